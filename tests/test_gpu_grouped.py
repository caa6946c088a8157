"""GPU parity of the m-target form (Sec. 3, Eq. (lanczos_blas3)) through the C
ABI: the Morton grouping bit for bit against the oracle's, the grouped block
Lanczos + eigensolve + forces against the oracle's grouped evaluation
(oracle.force_evaluation(group_m=m)), groups of one against the per-target
kernel, the MD step with grouping, and the capacity error of a union larger
than max_union.

Tolerances as in the per-target parity tests: forces 1e-6 eV/A (FP64) and
1e-3 eV/A (mixed), band energy 1e-8 / 1e-5 relative."""
import numpy as np
import pytest
import torch

import oracle
from oracle import density, grouping
from synth import CONFIGS, fcc_c60_crystal, workload_params

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(F=1e-6, Eb=1e-8, mom=1e-9), "mixed": dict(F=1e-3, Eb=1e-5, mom=1e-4)}


@pytest.fixture(scope="module")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    assert torch.cuda.is_available()
    return tb


def cfg_system(k, **over):
    cfg = CONFIGS[k]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"],
                                cfg["bridges"])
    p = workload_params(cfg, defl_tol=1e-9)
    p.update(over)
    return pos, L, p


_REF = {}


def grouped_oracle(key, pos, L, p, m, workers=1):
    if (key, m) not in _REF:
        _REF[(key, m)] = oracle.force_evaluation(pos, L, p, workers=workers, group_m=m)
    return _REF[(key, m)]


def run(tb, pos, L, p, prec, graph=False):
    s = tb.TBSystem(len(pos), L, p, prec=prec)
    s.set_positions(pos)
    if graph:
        s.capture()
        s.replay()
    else:
        s.evaluate()
    torch.cuda.synchronize()
    s.check()
    return s


def check_against(s, ref, p, prec):
    tol = TOL[prec]
    F = s.F.cpu().numpy()
    e = s.energies.cpu().numpy()
    errF = np.abs(F - ref.F).max()
    assert errF <= tol["F"], errF
    assert abs(e[0] - ref.E_band) <= tol["Eb"] * abs(ref.E_band)
    assert abs(e[5] - 4 * s.n) <= 1e-9 * s.n
    assert np.abs(F.sum(axis=0)).max() <= 1e-9 * s.n
    # per-target spectra through their quadrature moments (basis invariant)
    n, NT = s.n, s.NT
    lam = s.lam.cpu().numpy().reshape(n, NT)
    S = s.S.cpu().numpy().reshape(n, 4, NT)
    kd = s.kdim.cpu().numpy()
    for i in range(0, n, max(1, n // 97)):
        m = kd[i]
        assert m == ref.kdim[i], i
        w, wr = np.sum(S[i, :, :m] ** 2, axis=0), np.sum(ref.S[i] ** 2, axis=0)
        for q in range(2 * p["r"]):
            mg, mr = np.sum(w * lam[i, :m] ** q), np.sum(wr * ref.lam[i] ** q)
            assert abs(mg - mr) <= tol["mom"] * max(1.0, abs(mr)), (i, q)


@pytest.mark.parametrize("m", [2, 4])
@pytest.mark.parametrize("k", [0, 1])
def test_group_atoms_bit_exact(tb, k, m):
    # (an FP64 context holds W of 4m x 16 x max_union doubles in shared memory)
    pos, L, p = cfg_system(k, group_m=m, max_union=256)
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    s.set_positions(pos)
    s.group()
    torch.cuda.synchronize()
    s.check()
    ref = grouping.group_atoms(pos, L, m)
    g_off = s.g_off.cpu().numpy()
    g_idx = s.g_idx.cpu().numpy()
    assert len(g_off) == len(ref) + 1
    for q, grp in enumerate(ref):
        assert list(g_idx[g_off[q]:g_off[q + 1]]) == list(grp), q
    s.close()


def test_group_atoms_cell_edges(tb):
    """Coordinates on and just below a cell edge, and near the top of the box."""
    L = 8.0
    pos = np.full((16, 3), 1.0)
    pos[3] = [4.0, 1.0, 1.0]
    pos[9] = [3.9999999, 1.0, 1.0]
    pos[12] = [7.9999999999, 7.9, 7.9]
    pos[5] = [1.0, 5.0, 1.0]
    pos[7] = [np.nextafter(8.0, 0.0), 0.0, 0.0]
    p = workload_params(CONFIGS[0], group_m=2)
    s = tb.TBSystem(16, L, p, prec="fp64")
    s.set_positions(pos)
    s.group()
    torch.cuda.synchronize()
    assert list(s.g_idx.cpu().numpy()) == list(grouping.group_order(pos, L, 2))
    s.close()


@pytest.mark.parametrize("m", [2, 4])
@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_grouped_cfg0_matches_oracle(tb, prec, m):
    pos, L, p = cfg_system(0, group_m=m)
    ref = grouped_oracle("cfg0", pos, L, p, m)
    s = run(tb, pos, L, p, prec)
    check_against(s, ref, p, prec)
    s.close()


def test_grouped_ragged_last_group(tb):
    """Explicit groups of sizes 1, 2, 3 and 4 along the Morton order handed to
    the grouped entry point, against the oracle on the same groups."""
    pos, L, p = cfg_system(0, group_m=4)
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    s.set_positions(pos)
    s.neighbors()
    s.group()
    order = s.g_idx.cpu().numpy()
    sizes = [1, 2, 3, 4] * 24            # 240 atoms
    off = np.concatenate([[0], np.cumsum(sizes)]).astype(np.int32)
    s.n_groups = len(sizes)
    s.g_off = torch.tensor(off, device="cuda")
    s.assemble()
    s.krylov()
    s.find_mu(warm_start=False)
    s.forces()
    torch.cuda.synchronize()
    s.check()
    groups = [order[off[q]:off[q + 1]] for q in range(len(sizes))]
    ref = oracle.force_evaluation(pos, L, p, groups=groups)
    assert np.abs(s.F.cpu().numpy() - ref.F).max() <= TOL["fp64"]["F"]
    s.close()


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_singleton_groups_equal_the_per_target_kernel(tb, prec):
    pos, L, p = cfg_system(0, group_m=2)
    s = tb.TBSystem(len(pos), L, p, prec=prec)
    s.set_positions(pos)
    s.neighbors()
    s.assemble()
    n = len(pos)
    s.n_groups = n
    s.g_off = torch.arange(n + 1, dtype=torch.int32, device="cuda")
    s.g_idx = torch.arange(n, dtype=torch.int32, device="cuda")
    s.krylov()
    s.find_mu(warm_start=False)
    s.forces()
    torch.cuda.synchronize()
    s.check()
    F_g = s.F.cpu().numpy()
    s.close()
    p1 = dict(p, group_m=1)
    s1 = run(tb, pos, L, p1, prec)
    F_1 = s1.F.cpu().numpy()
    s1.close()
    assert np.abs(F_g - F_1).max() <= (1e-9 if prec == "fp64" else TOL["mixed"]["F"])


def test_grouped_full_size_benchmark_settings(tb):
    """1920-atom compressed cell, groups of four, the benchmark's Lanczos
    settings, CUDA-graph replay: every force against the oracle's grouped
    evaluation."""
    m = 4
    pos, L, p = cfg_system(1, group_m=m, max_union=320, reorth_passes=1, reorth_every=4)
    ref = grouped_oracle("cfg1", pos, L, p, m, workers=8)
    s = run(tb, pos, L, p, "mixed", graph=True)
    check_against(s, ref, p, "mixed")
    s.close()


def test_grouped_md_step_matches_evaluate(tb):
    """tb_md_step with group_m > 1 regroups and runs the grouped Krylov stage:
    its forces at the new positions equal a fresh grouped evaluation there."""
    from synth import maxwell_boltzmann_velocities
    pos, L, p = cfg_system(0, group_m=4)
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    s.set_positions(pos)
    s.vel.copy_(torch.as_tensor(maxwell_boltzmann_velocities(len(pos), 2000.0, 12.011, 5)))
    s.evaluate()
    for _ in range(3):
        s.md_step(0.5, 12.011)
    torch.cuda.synchronize()
    s.check()
    x = s.pos.cpu().numpy()
    F_md = s.F.cpu().numpy()
    s.close()
    s2 = run(tb, x, L, p, "fp64")
    # the step warm-starts mu from the previous one: equal up to the mu tolerance
    assert np.abs(F_md - s2.F.cpu().numpy()).max() <= 1e-8
    s2.close()


def test_union_capacity_is_reported(tb):
    pos, L, p = cfg_system(0, group_m=4, max_union=60)
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    s.set_positions(pos)
    s.evaluate()
    code, info = s.status()
    assert tb.binding.STATUS_NAMES[code] == "TB_ERR_CAPACITY" and info > 60
    s.close()


def test_grouped_entry_point_needs_group_contexts(tb):
    pos, L, p = cfg_system(0)
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    n = len(pos)
    with pytest.raises(tb.binding.TBError):
        tb.binding.tb_krylov_density_grouped(
            s.ctx, n, n, torch.arange(n + 1, dtype=torch.int32, device="cuda"),
            torch.arange(n, dtype=torch.int32, device="cuda"), s.c_off, s.c_idx, s.h_off,
            s.h_idx, s.Hblk, s.Hsk, s.lam, s.S, s.P, s.kdim)
    s.close()
