"""Writes chain_krylov_binomial.txt: the paper's closed form for the Krylov
vectors of the uniform chain (Sec. 3), H^r|0> = sum_k C(r,k) |2k - r>."""
import os
from math import comb

HERE = os.path.dirname(os.path.abspath(__file__))

if __name__ == "__main__":
    lines = ["# Sec. 3, one-dimensional uniform chain with t_{i,i+-1} = 1 and seed |0>:",
             "# H^r |0> = sum_{k=0}^{r} C(r,k) |2k - r>   (binomial coefficients; the paper's closed form)",
             "# columns: r  site(2k-r)  coefficient"]
    for r in range(0, 9):
        for k in range(r + 1):
            lines.append(f"{r} {2 * k - r} {comb(r, k)}")
    with open(os.path.join(HERE, "chain_krylov_binomial.txt"), "w") as fh:
        fh.write("\n".join(lines) + "\n")
