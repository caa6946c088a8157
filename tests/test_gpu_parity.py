"""GPU parity: the CUDA path against the FP64 CPU oracle on the same seeded
inputs, through the C ABI.

Tolerances (forces in eV/A, energies relative):
  FP64 path: forces <= 1e-6, band energy <= 1e-8;
  mixed path (FP32 sweeps/basis): forces <= 1e-3, band energy <= 1e-5;
  neighbour lists: bit-exact; electron count |N(mu) - N_e| <= 1e-9 N.
Spectra are compared through basis-invariant quantities (quadrature moments,
density-matrix blocks), since eigenvector signs and degenerate bases are free.
"""
import os

import numpy as np
import pytest
import torch

import oracle
from oracle import density, neighbors, hamiltonian, model
from synth import (CONFIGS, TB_CONSTANTS, workload_params, fcc_c60_crystal, linear_chain,
                   dimer)

pytestmark = pytest.mark.gpu

TOL = {"fp64": dict(F=1e-6, Eb=1e-8, rho=1e-7, mom=1e-9),
       "mixed": dict(F=1e-3, Eb=1e-5, rho=1e-3, mom=1e-4)}


@pytest.fixture(scope="session")
def tb():
    import __graft_entry__
    __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    assert torch.cuda.is_available()
    return tb


def cfg_system(k, ncell=None, **over):
    cfg = dict(CONFIGS[k])
    if ncell is not None:
        cfg["ncell"] = ncell
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"],
                                cfg["bridges"])
    p = workload_params(cfg, defl_tol=1e-9)
    p.update(over)
    return pos, L, p


_ORACLE = {}


def oracle_result(key, pos, L, p, workers=1):
    if key not in _ORACLE:
        _ORACLE[key] = oracle.force_evaluation(pos, L, p, workers=workers)
    return _ORACLE[key]


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


def gpu_records(s):
    n, NT = s.n, s.NT
    lam = s.lam.cpu().numpy().reshape(n, NT)
    S = s.S.cpu().numpy().reshape(n, 4, NT)
    P = s.P.cpu().numpy()
    kd = s.kdim.cpu().numpy()
    ho = s.h_off.cpu().numpy()
    recs = []
    for i in range(n):
        m = kd[i]
        deg = ho[i + 1] - ho[i]
        base = (i + ho[i]) * 4
        Pi = P[base * NT:(base + 4 * (deg + 1)) * NT].reshape(4 * (deg + 1), NT)
        recs.append((lam[i, :m], S[i, :, :m], Pi[:, :m]))
    return recs


def compare_full(tb, key, pos, L, p, prec, graph=False, workers=1):
    ref = oracle_result(key, pos, L, p, workers)
    s = run(tb, pos, L, p, prec, graph=graph)
    tol = TOL[prec]
    F = s.F.cpu().numpy()
    e = s.energies.cpu().numpy()
    errF = np.abs(F - ref.F).max()
    assert errF <= tol["F"], f"{key} {prec}: max |dF| {errF:.3e}"
    assert abs(e[0] - ref.E_band) <= tol["Eb"] * abs(ref.E_band)
    assert abs(e[3] - ref.E_rep) <= 1e-10 * abs(ref.E_rep)
    # electron count of the oracle's spectra at the GPU's mu
    lam_all = np.concatenate(ref.lam)
    w_all = np.concatenate([np.sum(S_ * S_, axis=0) for S_ in ref.S])
    mu_gpu = s.mu.cpu().item()
    n_at = density.electron_count(mu_gpu, lam_all, w_all, p["kT"])
    assert abs(n_at - 4 * len(pos)) <= (1e-9 if prec == "fp64" else 1e-5) * len(pos)
    assert abs(e[5] - 4 * len(pos)) <= 1e-9 * len(pos)
    assert np.abs(F.sum(axis=0)).max() <= 1e-9 * len(pos)
    return s, ref


# ---------------------------------------------------------------- lists

@pytest.mark.parametrize("k", [0, 1])
def test_neighbor_lists_bit_exact(tb, k):
    pos, L, p = cfg_system(k)
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    s.set_positions(pos)
    s.neighbors()
    torch.cuda.synchronize()
    s.check()
    hl, cl = s.lists()
    rh = neighbors.neighbor_lists(pos, L, p["rm"])
    rc = neighbors.cluster_lists(pos, L, p["Rc"])
    for i in range(len(pos)):
        assert np.array_equal(hl[i], rh[i]), i
        assert np.array_equal(cl[i], rc[i]), i


def test_neighbor_capacity_overflow_reports(tb):
    pos, L, p = cfg_system(0)
    p = dict(p, max_cluster=16)
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    s.set_positions(pos)
    s.neighbors()
    code, info = s.status()
    assert code == 4 and info > 16          # TB_ERR_CAPACITY, length needed


def test_position_outside_box_reports(tb):
    pos, L, p = cfg_system(0)
    pos = pos.copy()
    pos[7, 1] = L + 0.5
    s = tb.TBSystem(len(pos), L, p, prec="fp64")
    s.set_positions(pos)
    s.neighbors()
    code, info = s.status()
    assert code == 1 and info == 7          # TB_ERR_INVALID_ARG at atom 7


# ---------------------------------------------------------------- H blocks

def test_hamiltonian_blocks(tb):
    pos, L, p = cfg_system(0)
    s = tb.TBSystem(len(pos), L, p, prec="mixed")
    s.set_positions(pos)
    s.neighbors()
    s.assemble()
    torch.cuda.synchronize()
    s.check()
    hl = neighbors.neighbor_lists(pos, L, p["rm"])
    bonds = hamiltonian.BondTable(pos, L, hl, p)
    nb = len(bonds.src)
    H = s.Hblk.cpu().numpy()[:nb * 16].reshape(nb, 4, 4)
    G = s.dHblk.cpu().numpy()[:nb * 48].reshape(nb, 3, 4, 4)
    rec = s.Hsk.cpu().numpy()[:nb * 4].reshape(nb, 4).astype(np.float64)
    assert np.abs(H - bonds.t).max() <= 1e-12
    assert np.abs(G - bonds.g).max() <= 1e-11
    # FP32 record (s(r), l): the block it stands for is s(r) SK(l), and l is d/|d|
    r_b = np.linalg.norm(bonds.d, axis=1)
    assert np.abs(rec[:, 0] - model.hopping_scale(r_b, p)[0]).max() <= 1e-6
    assert np.abs(rec[:, 1:] - bonds.d / r_b[:, None]).max() <= 1e-6
    blocks = np.stack([rec[b, 0] * model.sk_matrix(rec[b, 1:], p) for b in range(nb)])
    assert np.abs(blocks - bonds.t).max() <= 1e-5


# ---------------------------------------------------------------- spectral records

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_spectral_record_moments_and_rho(tb, prec):
    pos, L, p = cfg_system(0)
    ref = oracle_result("cfg0", pos, L, p)
    s = run(tb, pos, L, p, prec)
    recs = gpu_records(s)
    tol = TOL[prec]
    kT = p["kT"]
    for i in range(0, len(pos), 7):
        lam, S, P = recs[i]
        assert len(lam) == ref.kdim[i]
        w, wr = np.sum(S * S, axis=0), np.sum(ref.S[i] ** 2, axis=0)
        for q in range(2 * p["r"]):
            mg, mr = np.sum(w * lam ** q), np.sum(wr * ref.lam[i] ** q)
            assert abs(mg - mr) <= tol["mom"] * max(1.0, abs(mr)), (i, q)
        f = density.fermi((lam - ref.mu) / kT)
        rg = (P * f) @ S.T
        rr = density.rho_blocks(ref.S[i], ref.P[i], ref.lam[i], ref.mu, kT).reshape(-1, 4)
        assert np.abs(rg - rr).max() <= tol["rho"], i


# ---------------------------------------------------------------- full evaluation

@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_forces_cfg0(tb, prec):
    pos, L, p = cfg_system(0)
    compare_full(tb, "cfg0", pos, L, p, prec)


@pytest.mark.parametrize("prec", ["fp64", "mixed"])
def test_forces_cfg1_full_size_graph(tb, prec):
    """1920-atom compressed cell at full size, CUDA-graph replay as benchmarked."""
    pos, L, p = cfg_system(1)
    compare_full(tb, "cfg1", pos, L, p, prec, graph=True, workers=8)


def test_benchmark_configuration_full_size(tb):
    """The benchmark's settings on the 1920-atom cell: one classical
    Gram-Schmidt pass, full reorthogonalisation every fourth Lanczos step
    (the steps between project out the last two blocks only)."""
    pos, L, p = cfg_system(1)
    compare_full(tb, "cfg1", pos, L, dict(p, reorth_passes=1, reorth_every=4), "mixed",
                 graph=True, workers=8)


def test_forces_bridged_uneven_clusters(tb):
    pos, L, p = cfg_system(2, ncell=2, r=10)
    s, ref = compare_full(tb, "cfg2small", pos, L, p, "fp64")
    sizes = np.diff(s.c_off.cpu().numpy())
    assert sizes.max() - sizes.min() >= 20


@pytest.mark.parametrize("schedule", ["persistent", "separate"])
def test_schedules_match(tb, schedule):
    """Mixed path: one persistent launch that queues the Krylov targets and
    then the group eigensolves, or separate Krylov and eigensolver launches:
    the same answers within the path's tolerance, and the oracle's."""
    pos, L, p = cfg_system(0)
    s_alt, _ = compare_full(tb, "cfg0", pos, L, dict(p, schedule=schedule), "mixed")
    s_def, _ = compare_full(tb, "cfg0", pos, L, p, "mixed")
    assert np.abs(s_alt.F.cpu().numpy() - s_def.F.cpu().numpy()).max() <= TOL["mixed"]["F"]


def test_single_reorth_pass_within_tolerance(tb):
    pos, L, p = cfg_system(0)
    compare_full(tb, "cfg0", pos, L, dict(p, reorth_passes=1), "fp64")


def test_graph_replay_is_deterministic(tb):
    pos, L, p = cfg_system(0)
    s = run(tb, pos, L, p, "mixed", graph=True)
    F1 = s.F.clone()
    s.replay()
    s.replay()
    torch.cuda.synchronize()
    assert torch.equal(F1, s.F)
    s2 = run(tb, pos, L, p, "mixed")
    assert torch.equal(F1, s2.F)


# ---------------------------------------------------------------- edge cases

def test_dimer(tb):
    pos, L = dimer(1.42)
    p = dict(TB_CONSTANTS, kT=0.1, Rc=5.0, r=3, defl_tol=1e-9, n_electrons_per_atom=4.0,
             max_cluster=8)
    compare_full(tb, "dimer", pos, L, p, "fp64")


def test_isolated_atom_and_pair(tb):
    pos = np.array([[1.0, 1.0, 1.0], [10.0, 10.0, 10.0], [11.4, 10.0, 10.0]])
    L = 20.0
    p = dict(TB_CONSTANTS, kT=0.1, Rc=5.0, r=4, defl_tol=1e-9, n_electrons_per_atom=4.0,
             max_cluster=8)
    s, ref = compare_full(tb, "iso", pos, L, p, "fp64")
    assert s.kdim.cpu().numpy()[0] == 4


def test_chain_deflation_and_half_filling(tb):
    p = dict(TB_CONSTANTS, Es=0.0, Ep=0.0, Vss=1.0, Vsp=0.0, Vpps=0.0, Vppp=0.0, kT=0.1,
             Rc=8.0, r=5, defl_tol=1e-9, n_electrons_per_atom=4.0, max_cluster=16)
    pos, L = linear_chain(24, p["r0"])
    s, ref = compare_full(tb, "chain", pos, L, p, "fp64")
    kd = s.kdim.cpu().numpy()
    assert np.all(kd == 4 + (p["r"] - 1)) and np.all(kd == ref.kdim)
    assert abs(s.mu.cpu().item()) < 1e-9
    s2, _ = compare_full(tb, "chain", pos, L, dict(p, defl_tol=1e-4), "mixed")
    assert np.all(s2.kdim.cpu().numpy() == kd)


def test_krylov_order_one(tb):
    pos, L, p = cfg_system(0)
    p = dict(p, r=1)
    compare_full(tb, "cfg0_r1", pos, L, p, "fp64")


# ---------------------------------------------------------------- MD

def test_md_step_matches_oracle_verlet(tb):
    from synth import maxwell_boltzmann_velocities
    from oracle import md
    pos, L, p = cfg_system(0)
    vel = maxwell_boltzmann_velocities(len(pos), 2000.0, 12.011, seed=5)
    s = run(tb, pos, L, p, "fp64")
    s.vel.copy_(torch.as_tensor(vel))
    for _ in range(2):
        s.md_step(0.5, 12.011)
    torch.cuda.synchronize()
    s.check()

    def ffn(x):
        r = oracle.force_evaluation(x, L, p)
        return r.F, r.E_total
    x, v = pos.copy(), vel.copy()
    F = oracle_result("cfg0", pos, L, p).F
    for _ in range(2):
        x, v, F, epot = md.verlet_step(x, v, F, L, 0.5, 12.011, ffn)
    dx = s.pos.cpu().numpy() - x
    dx -= L * np.rint(dx / L)
    assert np.abs(dx).max() <= 1e-9
    assert np.abs(s.vel.cpu().numpy() - v).max() <= 1e-9
    e = s.energies.cpu().numpy()
    assert abs(e[4] - epot) <= 1e-8 * abs(epot)
    assert abs(e[7] - md.kinetic_energy(v, 12.011)) <= 1e-9 * abs(e[7])


def test_kernels_per_evaluation_count(tb):
    """The library's own count of kernels per force evaluation on the 1920-atom
    cell (cell lists: 6; assembly; Krylov with the eigensolve inside in the
    mixed path, separate group eigensolver + refinement in FP64; mu; 3 for
    density blocks, bond forces, and per-atom sums with the energies)."""
    pos, L, p = cfg_system(1)
    counts = {}
    for prec in ("mixed", "fp64"):
        s = tb.TBSystem(len(pos), L, p, prec=prec)
        counts[prec] = tb.binding.tb_ctx_kernels_per_evaluation(s.ctx, len(pos), L)
        s.close()
    assert counts == {"mixed": 12, "fp64": 14}
    s = tb.TBSystem(len(pos), L, dict(p, schedule="separate"), prec="mixed")
    assert tb.binding.tb_ctx_kernels_per_evaluation(s.ctx, len(pos), L) == 13
    s.close()
