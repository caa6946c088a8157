// Distance scaling of the tight-binding model (Eq. (1), Xu's functional form
// named in Sec. 5): A (r_ref/r)^e exp{e[-(r/r_cut)^ec + (r_ref/r_cut)^ec]}
// for r < r1, a C1 cubic tail on [r1, rm] reaching zero with zero slope at rm,
// and zero beyond.
#pragma once
#include <cmath>
#include "tb.h"

struct tb_gsp {
  double A, rref, e, rcut, ec;   // GSP form
  double r1, rm;                 // tail interval
  double v1, d1, ta, tb;         // tail: v1 + d1 x + ta x^2 + tb x^3, x = r - r1
  double lrref, lrcut, C;        // ln r_ref, ln r_cut, (r_ref/r_cut)^ec
};

// The GSP form through logarithms: with p = (r/r_cut)^ec = exp(ec (ln r - ln r_cut)),
// v = A exp{e [ln r_ref - ln r - p + C]} and dv/dr = -v e (1 + ec p) / r: one
// logarithm and two exponentials (FP64 transcendentals are costly on this GPU;
// the power form takes two powers and an exponential).
__host__ __device__ inline void tb_gsp_core(const tb_gsp& g, double r, double& v,
                                            double& dv) {
  const double lr = log(r);
  const double pr = exp(g.ec * (lr - g.lrcut));
  v = g.A * exp(g.e * (g.lrref - lr - pr + g.C));
  dv = -v * g.e * (1.0 + g.ec * pr) / r;
}

inline tb_gsp tb_make_gsp(double A, double rref, double e, double rcut, double ec,
                          double r1, double rm) {
  tb_gsp g{A, rref, e, rcut, ec, r1, rm, 0, 0, 0, 0, std::log(rref), std::log(rcut),
           std::pow(rref / rcut, ec)};
  tb_gsp_core(g, r1, g.v1, g.d1);
  const double dl = rm - r1;
  g.ta = -(3.0 * g.v1 + 2.0 * g.d1 * dl) / (dl * dl);
  g.tb = (2.0 * g.v1 + g.d1 * dl) / (dl * dl * dl);
  return g;
}

__device__ inline void tb_gsp_eval(const tb_gsp& g, double r, double& v, double& dv) {
  if (r < g.r1) {
    tb_gsp_core(g, r, v, dv);
  } else if (r < g.rm) {
    double x = r - g.r1;
    v = g.v1 + x * (g.d1 + x * (g.ta + x * g.tb));
    dv = g.d1 + x * (2.0 * g.ta + 3.0 * x * g.tb);
  } else {
    v = 0.0;
    dv = 0.0;
  }
}

inline tb_gsp tb_hopping_gsp(const tb_params& p) {
  return tb_make_gsp(1.0, p.r0, p.n, p.rc, p.nc, p.r1, p.rm);
}
inline tb_gsp tb_repulsion_gsp(const tb_params& p) {
  return tb_make_gsp(p.phi0, p.d0, p.m, p.dc, p.mc, p.r1, p.rm);
}
