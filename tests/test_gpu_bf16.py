"""BF16 H.V sweeps (Slater-Koster records and the Krylov block V_k rounded to
BF16 in the sweep's products, FP32 accumulation, the rest as the mixed path)
against the FP64 oracle.

BF16 keeps 8 significant bits (unit roundoff 2^-9 ~ 2e-3), so every sweep
perturbs H V by ~2e-3 relative; the block recursion then projects a slightly
different operator and the forces move by a few hundredths of an eV/A at
most-affected atoms.  The 1e-3 eV/A bar of the mixed path is not met, and this
test records that: what holds is the electron count (mu is solved exactly on
the BF16 record), Newton's third law (the force is a sum of pair terms), the
band energy to 1e-4 relative and the forces to 0.5 eV/A (max) and 0.1 eV/A
(rms).  The mixed FP32 sweep on the same cell stays within 1e-3.
"""
import numpy as np
import pytest
import torch

import oracle
from synth import CONFIGS, fcc_c60_crystal, workload_params

pytestmark = pytest.mark.gpu


@pytest.fixture(scope="module")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    assert torch.cuda.is_available()
    return tb


@pytest.mark.parametrize("k", [0, 1])
def test_bf16_sweep_error_against_oracle(tb, k):
    cfg = CONFIGS[k]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"])
    p = workload_params(cfg, defl_tol=1e-9)
    ref = oracle.force_evaluation(pos, L, p, workers=8)
    errs = {}
    for prec in ("bf16", "mixed"):
        s = tb.TBSystem(len(pos), L, p, prec=prec)
        s.set_positions(pos)
        s.capture()
        s.replay()
        torch.cuda.synchronize()
        s.check()
        F = s.F.cpu().numpy()
        e = s.energies.cpu().numpy()
        dF = np.abs(F - ref.F)
        errs[prec] = (dF.max(), np.sqrt(np.mean(dF ** 2)), abs(e[0] - ref.E_band) / abs(ref.E_band))
        assert abs(e[5] - 4 * s.n) <= 1e-9 * s.n
        assert np.abs(F.sum(axis=0)).max() <= 1e-9 * s.n
        s.close()
    fmax, frms, eb = errs["bf16"]
    print(f"cfg{k} BF16 sweep vs FP64 oracle: max |dF| {fmax:.3e}, rms {frms:.3e} eV/A, "
          f"band energy {eb:.2e} relative; FP32 sweep: max |dF| {errs['mixed'][0]:.2e}")
    assert fmax <= 0.5 and frms <= 0.1 and eb <= 1e-4
    assert errs["mixed"][0] <= 1e-3 and errs["mixed"][2] <= 1e-5


def test_bf16_overflow_records_long_range(tb):
    """The long-range 240-atom cell (hoppings to 7.0 A): no target's records
    fit shared memory, so every sweep gathers them from the bond table by
    index and rounds them to BF16 there.  Same bars as above, and the mixed
    path's FP32 gather within 1e-3."""
    from synth import LONGRANGE
    cfg = LONGRANGE[0]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"],
                                cfg["bridges"])
    p = workload_params(cfg, defl_tol=1e-9)
    ref = oracle.force_evaluation(pos, L, p, workers=8)
    errs = {}
    for prec in ("bf16", "mixed"):
        s = tb.TBSystem(len(pos), L, p, prec=prec)
        s.set_positions(pos)
        s.capture()
        s.replay()
        torch.cuda.synchronize()
        s.check()
        F = s.F.cpu().numpy()
        e = s.energies.cpu().numpy()
        dF = np.abs(F - ref.F)
        errs[prec] = (dF.max(), np.sqrt(np.mean(dF ** 2)), abs(e[0] - ref.E_band) / abs(ref.E_band))
        assert abs(e[5] - 4 * s.n) <= 1e-9 * s.n
        assert np.abs(F.sum(axis=0)).max() <= 1e-9 * s.n
        s.close()
    fmax, frms, eb = errs["bf16"]
    print(f"long-range 240 BF16 sweep vs FP64 oracle: max |dF| {fmax:.3e}, rms {frms:.3e} eV/A, "
          f"band energy {eb:.2e} relative; FP32 sweep: max |dF| {errs['mixed'][0]:.2e}")
    assert fmax <= 0.5 and frms <= 0.1 and eb <= 1e-4
    assert errs["mixed"][0] <= 1e-3 and errs["mixed"][2] <= 1e-5
