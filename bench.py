#!/usr/bin/env python
"""Benchmark: atom force evaluations per second on the 1920-atom compressed
fcc C60 cell (2x2x2 supercell at a = 13.0 A, cluster cutoff 6.0 A, Krylov block
order r = 12), one full force evaluation (lists, Hamiltonian blocks, block
Lanczos, projected eigensolve, mu, density blocks, forces) per step, replayed
as one CUDA graph.

  python bench.py [--gpus N] [--steps K] [--warmup W] [--prec mixed|fp64]
                  [--impl ours|reference]
                  [--workload c60_1920|bridged6480|longrange1920|md15360|npt15360|
                              autograd1920|diamond_eos] [--no-autotune]

Before the timed region the library's autotuner (tb_autotune) times the launch
plans of the mixed path's block-Lanczos stage on the workload's lists
(persistent Krylov + eigensolve queue in index order or largest clusters first,
separate launches, separate launches per cluster-size bucket with per-bucket
tiles) and the timed steps replay the fastest; the line reports the
cluster-size histogram and the choices ("autotune").

--workload bridged6480 is the uneven-cluster workload: the 3x3x3 fcc C60 cell
(6480 atoms, a = 12.5 A) with 30% of the nearest-neighbour molecule pairs
bridged by 1.55-1.65 A inter-cage contacts, 0.08 A jitter, cluster cutoff
6.5 A, r = 16, cluster capacity 384; the accuracy and CPU baseline come from a
bounded oracle sample (the spectral records of a few targets).

--workload longrange1920 is the same measurement in the long-range
(dense-Hamiltonian) regime: synthetic hoppings of Xu's functional form decaying
slowly to a 7.0 A cutoff (H lists of 149-172 atoms), cluster cutoff 8.0 A
(219-243 atoms per cluster), r = 12, on the same 1920-atom cell.  The CPU
baseline and the accuracy figures come from a bounded oracle sample (the bond
table of a few targets' clusters and those targets' spectral records).

--workload md15360 times molecular dynamics instead: the 4x4x4 fcc C60 cell
of 15360 atoms (a = 12.5 A, cluster cutoff 6.5 A, r = 16), velocity-Verlet
steps of 0.5 fs from 2000 K Maxwell-Boltzmann velocities, one CUDA graph per
step; value = atom-steps/s, with the NVE energy drift of the mixed and FP64
paths over the same steps from the same state.

--workload npt15360 times NPT molecular dynamics of the same 15360-atom cell at
the paper's C60 polymerisation conditions (25 GPa, 500 K): each step is one
velocity-Verlet step, its virial and a weak-coupling (Berendsen) scaling of the
velocities, positions and box; value = atom-steps/s, with the temperature,
pressure and box over the timed steps.

--workload autograd1920 times the exact local gradient instead (the
truncated local free energy at Krylov order r = r_min, whose projected
problem is the dense cluster eigenproblem, ~392 x 392 per target, with its
Daleckii-Krein backward) on the 1920-atom compressed cell: one step = forward
(spectra, mu, energies) + backward; the stored-eigenvector backward is timed
against the recomputing one, and --fd-coords seeded coordinates are checked
by central differences (h = 1e-4 A) of the FP64 energy.

--workload diamond_eos times pressure evaluations of the 4x4x4 cubic diamond
supercell (512 atoms; Sec. 5's equation-of-state workload): one step = one
force evaluation plus the virial pressure at one lattice constant, cycling
through eight lattice constants; it reports the equation of state E(V), P(V),
a Birch-Murnaghan fit, and its convergence with the block order r and with the
8x8x8 supercell (4096 atoms).

Prints one JSON line (rank 0).  With --gpus N > 1 (torchrun, one rank per GPU)
every rank evaluates its own replica of the cell; value = total atoms / max time.
--impl reference times the FP64 CPU oracle on a bounded sample of the same
workload on the host cores.
"""
import argparse
import hashlib
import json
import os
import statistics
import subprocess
import sys
import tempfile
import time

ROOT = os.path.dirname(os.path.abspath(__file__))
sys.path.insert(0, ROOT)

METRIC = ("atom force evals/s (batched mixed vs plain FP64, 1 GB300) at "
          "≤1e-3 eV/Å error")
UNIT = "atom force evals/s"
CONFIG_INDEX = 1


def parse():
    ap = argparse.ArgumentParser()
    ap.add_argument("--gpus", type=int, default=1)
    ap.add_argument("--steps", type=int, default=500)
    ap.add_argument("--warmup", type=int, default=5)
    ap.add_argument("--impl", default="ours", choices=["ours", "reference"])
    ap.add_argument("--prec", default="mixed", choices=["mixed", "fp64", "bf16"])
    ap.add_argument("--no-cpu-baseline", action="store_true")
    ap.add_argument("--reorth-passes", type=int, default=1)
    ap.add_argument("--reorth-every", type=int, default=4)
    ap.add_argument("--workload", default="c60_1920",
                    choices=["c60_1920", "bridged6480", "longrange1920", "md15360", "npt15360",
                             "autograd1920", "diamond_eos"])
    ap.add_argument("--fd-coords", type=int, default=8)
    ap.add_argument("--no-autotune", action="store_true",
                    help="keep the library's default launch plan (no tb_autotune)")
    ap.add_argument("--schedule", default="auto",
                    choices=["auto", "persistent", "persistent_largest_first", "separate",
                             "bucketed"],
                    help="launch plan of the mixed block-Lanczos stage (auto: the tuned one)")
    ap.add_argument("--no-fp64-compare", action="store_true")
    ap.add_argument("--group-m", type=int, default=1,
                    help="targets per group of the m-target form (1 = per-target clusters)")
    ap.add_argument("--max-union", type=int, default=320,
                    help="union-cluster capacity of the m-target form")
    return ap.parse_args()


def workload(name="c60_1920"):
    from synth import CONFIGS, LONGRANGE, fcc_c60_crystal, workload_params
    cfg = (LONGRANGE[1] if name == "longrange1920" else
           CONFIGS[2] if name == "bridged6480" else CONFIGS[CONFIG_INDEX])
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"],
                                cfg["bridges"])
    p = workload_params(cfg, defl_tol=1e-9)
    return cfg, pos, L, p


def list_launches(L, Rc):
    """Kernels of one list build: cell lists (binning, scan, fill, search, scan,
    compaction, plus the position check) when the box holds >= 3 cells of side
    Rc + 0.01 A per dimension, else the brute-force count/scan/fill."""
    return 7 if int(L / (Rc + 0.01)) >= 3 else 4


L2_NOTE = ("L2 flushed between timed steps on the GPU (256 MB write); the oracle arm "
           "runs on the host")


def config_dict(cfg, n, world=1, extra=None):
    """The workload, identical for the GPU arm and the oracle (reference) arm;
    run settings of one arm go to the line's "run" key instead."""
    d = {"workload": cfg["name"], "n_atoms": n, "a": cfg["a"], "ncell": cfg["ncell"],
         "Rc": cfg["Rc"], "krylov_r": cfg["r"], "kT": cfg["kT"], "l2": L2_NOTE,
         "parallelism": f"replicas x{world}" if world > 1 else "single GPU"}
    if cfg.get("model") == "longrange":
        d.update(model="synthetic long-range GSP hoppings (nc 2, rc 4.0 A, tail 6.5-7.0 A)",
                 rm=7.0, max_hnbr=cfg["max_hnbr"], max_cluster=cfg["max_cluster"])
    if extra:
        d.update(extra)
    return d


# ---------------------------------------------------------------- ranks

def max_over_ranks(x, world, device):
    """The largest of one float over the ranks of the job (the job's time is
    its slowest rank's); the value itself for a single rank."""
    if world <= 1:
        return x
    import torch
    import torch.distributed as dist
    t = torch.tensor([float(x)], dtype=torch.float64, device=device)
    dist.all_reduce(t, op=dist.ReduceOp.MAX)
    return t.item()


def job_throughput(units_per_rank, world, steps, total_ms):
    """Whole-job rate: every rank processes units_per_rank per step (replicas,
    weak scaling) and the job takes the slowest rank's total_ms."""
    return world * units_per_rank * steps / (total_ms / 1e3)


# ---------------------------------------------------------------- CPU oracle

def time_oracle_full(pos, L, p):
    """One full oracle force evaluation, single process (the m-target form when
    p holds group_m > 1)."""
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    import oracle
    t0 = time.perf_counter()
    res = oracle.force_evaluation(pos, L, p, group_m=p.get("group_m", 1))
    return time.perf_counter() - t0, res


def oracle_sample_step(ctxd, stride=10):
    """Per-target oracle work (cluster H, block Lanczos, eigenpairs, density
    blocks at a fixed mu) for every `stride`-th target."""
    from oracle.pipeline import target_record
    from oracle.density import rho_blocks
    p = ctxd["p"]
    t0 = time.perf_counter()
    nt = 0
    for i in range(0, len(ctxd["pos"]), stride):
        lam, S, P = target_record(ctxd["bonds"], ctxd["cl"][i], ctxd["hl"][i], p["r"],
                                  p["defl_tol"])
        rho_blocks(S, P, lam, 4.5, p["kT"])
        nt += 1
    return nt, time.perf_counter() - t0


def oracle_target_sample(pos, L, p, k=4):
    """The oracle's pieces of one force evaluation on a bounded sample: the
    bond table (hopping blocks and their gradients) of every atom in the
    clusters of the first k targets, then those targets' records (cluster H,
    block Lanczos, eigenpairs, density blocks at a fixed mu).  Returns the
    seconds per atom (bond rows per atom + record per target), the number of
    atoms whose bond rows were built, and the records."""
    from oracle.neighbors import neighbor_lists, cluster_lists
    from oracle.hamiltonian import BondTable
    from oracle.pipeline import target_record
    from oracle.density import rho_blocks
    hl = neighbor_lists(pos, L, p["rm"])
    cl = cluster_lists(pos, L, p["Rc"])
    targets = list(range(k))
    union = set()
    for i in targets:
        union |= set(int(x) for x in cl[i])
    hl_sub = [hl[i] if i in union else hl[i][:0] for i in range(len(pos))]
    t0 = time.perf_counter()
    bonds = BondTable(pos, L, hl_sub, p)
    t_b = time.perf_counter() - t0
    t0 = time.perf_counter()
    recs = []
    for i in targets:
        lam, S, P = target_record(bonds, cl[i], hl[i], p["r"], p["defl_tol"])
        rho_blocks(S, P, lam, 3.4, p["kT"])
        recs.append((i, lam, S))
    t_t = time.perf_counter() - t0
    return t_b / len(union) + t_t / k, len(union), recs


def sampled_moment_error(system, recs, r):
    """Largest relative difference of the quadrature moments sum_k w_k lam_k^q
    (q < 2r) between the library's spectral records and the oracle's for the
    sampled targets (basis-invariant)."""
    import numpy as np
    n, NT = system.n, system.NT
    lam = system.lam.cpu().numpy().reshape(n, NT)
    S = system.S.cpu().numpy().reshape(n, 4, NT)
    kd = system.kdim.cpu().numpy()
    err = 0.0
    for i, lr, Sr in recs:
        m = kd[i]
        w, wr = np.sum(S[i, :, :m] ** 2, axis=0), np.sum(Sr ** 2, axis=0)
        for q in range(2 * r):
            mg, mr = np.sum(w * lam[i, :m] ** q), np.sum(wr * lr ** q)
            err = max(err, abs(mg - mr) / max(1.0, abs(mr)))
    return err


def run_reference(args):
    rank = int(os.environ.get("RANK", "0"))
    if rank != 0:
        return 0
    os.environ.setdefault("OMP_NUM_THREADS", "1")
    os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
    cfg, pos, L, p = workload(args.workload)
    if cfg.get("model") == "longrange" or args.workload == "bridged6480":
        for _ in range(args.warmup):
            oracle_target_sample(pos, L, p, k=2)
        per_atom = []
        for _ in range(args.steps):
            t, nu, _ = oracle_target_sample(pos, L, p, k=2)
            per_atom.append(t)
        value = 1.0 / statistics.mean(per_atom)
        sample = (f"per step: the bond table of the {nu} atoms in the clusters of 2 targets "
                  f"and those targets' records; value = 1 / (bond-table seconds per atom + "
                  f"record seconds per target)")
        line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * statistics.mean(per_atom) * len(pos),
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": config_dict(cfg, len(pos), int(os.environ.get("WORLD_SIZE", "1"))),
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": sample},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    from oracle.neighbors import neighbor_lists, cluster_lists
    from oracle.hamiltonian import BondTable
    hl = neighbor_lists(pos, L, p["rm"])
    cl = cluster_lists(pos, L, p["Rc"])
    ctxd = dict(pos=pos, p=p, hl=hl, cl=cl, bonds=BondTable(pos, L, hl, p))
    for _ in range(args.warmup):
        oracle_sample_step(ctxd)
    tot_t, tot_n = 0.0, 0
    for _ in range(args.steps):
        nt, dt = oracle_sample_step(ctxd)
        tot_t += dt
        tot_n += nt
    value = tot_n / tot_t
    sample = (f"per step: cluster H, block Lanczos, eigenpairs and density blocks of "
              f"{tot_n // args.steps} of the {len(pos)} targets (every 10th); lists and "
              f"bond table built once outside the timed region")
    line = {"metric": METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
            "steps": args.steps, "warmup": args.warmup,
            "ms_per_step": 1e3 * tot_t / args.steps, "higher_is_better": True,
            "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
            "impl": "reference",
            "config": config_dict(cfg, len(pos), int(os.environ.get("WORLD_SIZE", "1"))),
            "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                             "sample": sample},
            "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                    "d2h_bytes_per_step": 0}}
    print(json.dumps(line), flush=True)
    return 0


# ---------------------------------------------------------------- clocks

class ClockSampler:
    Q = ("index,clocks.sm,clocks.max.sm,power.draw,clocks_event_reasons.active,"
         "clocks_event_reasons.hw_slowdown,clocks_event_reasons.hw_thermal_slowdown,"
         "clocks_event_reasons.sw_thermal_slowdown,clocks_event_reasons.sw_power_cap")

    def __init__(self, index):
        self.index = index
        self.f = tempfile.NamedTemporaryFile(mode="w+", suffix=".csv", delete=False)
        try:
            self.p = subprocess.Popen(
                ["nvidia-smi", f"--query-gpu={self.Q}", "--format=csv,noheader,nounits",
                 "-i", str(index), "-lms", "200"], stdout=self.f, stderr=subprocess.DEVNULL)
        except OSError:
            self.p = None

    def stop(self):
        if self.p is None:
            return None
        time.sleep(0.3)
        self.p.terminate()
        self.p.wait(timeout=10)
        self.f.flush()
        rows = [r.split(",") for r in open(self.f.name).read().strip().splitlines() if r]
        os.unlink(self.f.name)
        sm, mx, reasons = [], [], set()
        names = ["hw_slowdown", "hw_thermal_slowdown", "sw_thermal_slowdown", "sw_power_cap"]
        for r in rows:
            try:
                sm.append(float(r[1]))
                mx.append(float(r[2]))
                for nm, v in zip(names, r[5:9]):
                    if v.strip().lower() == "active":
                        reasons.add(nm)
            except (ValueError, IndexError):
                continue
        if not sm:
            return None
        return {"sm_mhz": statistics.median(sm), "sm_max_mhz": max(mx),
                "reasons": sorted(reasons), "samples": len(sm)}


# ---------------------------------------------------------------- our path

def algorithmic_sweep_bytes(system, prec):
    """Bytes per Krylov launch of the H.V sweeps: per target and sweep
    nnzb*(16 b_H + 4) + 2*(4 n_c * 4 b_V), times r sweeps, summed over targets."""
    import numpy as np
    hl, cl = system.lists()
    n = system.n
    bH = 8 if prec == "fp64" else 4
    r = system.tp.r
    total = 0
    hsets = [set(x.tolist()) for x in hl]
    for i in range(n):
        c = cl[i]
        cs = set(c.tolist())
        nnzb = len(c) + sum(len(hsets[a] & cs) for a in c)
        total += r * (nnzb * (16 * bH + 4) + 2 * (4 * len(c) * 4 * bH))
    return total


def algorithmic_sweep_bytes_grouped(system, prec):
    """Bytes per grouped Krylov launch of the H.V sweeps: per group and sweep
    nnzb_u*(16 b_H + 4) + 2*(4 n_u * 4 m_g * b_V) over the union cluster u of the
    group's m_g targets (H read once for all of them), times r sweeps."""
    hl, cl = system.lists()
    g_off = system.g_off.cpu().numpy()
    g_idx = system.g_idx.cpu().numpy()
    bH = 8 if prec == "fp64" else 4
    r = system.tp.r
    hsets = [set(x.tolist()) for x in hl]
    total = 0
    for q in range(len(g_off) - 1):
        mem = g_idx[g_off[q]:g_off[q + 1]]
        u = set()
        for i in mem:
            u |= set(cl[i].tolist())
        nnzb = len(u) + sum(len(hsets[a] & u) for a in u)
        total += r * (nnzb * (16 * bH + 4) + 2 * (4 * len(u) * 4 * len(mem) * bH))
    return total


def record_bytes(system, prec):
    """Bytes per launch of the spectral records between the block Lanczos and
    the projected eigensolve, and of the eigensolve's outputs, for the
    persistent kernel that does both: per target T written and read
    (2 NT^2 * 8), the Y rows written and read (2 * 4(deg+1) NT * b_V),
    lambda and S (5 NT * 8) and P (4(deg+1) NT * 8)."""
    hl, _ = system.lists()
    NT = system.NT
    bV = 8 if prec == "fp64" else 4
    total = 0
    for x in hl:
        rows = 4 * (len(x) + 1)
        total += 2 * NT * NT * 8 + 2 * rows * NT * bV + 5 * NT * 8 + rows * NT * 8
    return total


def kernel_traffic(prec, name="krylov_traffic.json", workload=None):
    """DRAM bytes per Krylov launch from the committed ncu summary, or None if
    the kernel source changed since it was taken or the summary is of another
    workload."""
    path = os.path.join(ROOT, "profiles", name)
    if not os.path.exists(path):
        return None
    rec = json.load(open(path))
    if workload is not None and not rec.get("workload", "").startswith(workload):
        return None
    h = hashlib.sha256()
    for rel in rec.get("sources", []):
        src = os.path.join(ROOT, rel)
        if not os.path.exists(src):           # a source of that kernel is gone: changed
            return None
        h.update(open(src, "rb").read())
    if not rec.get("sources") or rec.get("source_sha256") != h.hexdigest():
        return None
    return rec.get("dram_bytes_per_launch", {}).get(prec)


def timed_leg(system, steps, flush, stream, B):
    """Mean ms per graph replay (L2 flushed before each) and mean stage times
    of `steps` replays of an already captured system."""
    import torch
    for _ in range(3):
        system.replay()
    torch.cuda.synchronize()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    tot, st = 0.0, {k: [] for k in B.STAGES}
    for k in range(steps):
        flush.fill_(float(k))
        e0.record(stream)
        system.replay()
        e1.record(stream)
        e1.synchronize()
        tot += e0.elapsed_time(e1)
        for name, v in B.tb_profile_read(system.ctx).items():
            if v >= 0:
                st[name].append(v)
    system.check()
    return tot / steps, {k: statistics.mean(v) for k, v in st.items() if v}


def kernel_traffic_record(prec, name, workload):
    """{"dram": bytes, "l2": bytes} per launch of the dominant kernel from the
    committed ncu record, or None if stale or of another workload."""
    d = kernel_traffic(prec, name, workload)
    if d is None:
        return None
    rec = json.load(open(os.path.join(ROOT, "profiles", name)))
    return {"dram": d, "l2": rec.get("l2_bytes_per_launch", {}).get(prec)}


def run_ours(args):
    import torch
    import __graft_entry__
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if world > 1 and rank == 0:
        __graft_entry__.build()
    if world > 1:
        import torch.distributed as dist
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        dist.barrier()
        if rank != 0:
            __graft_entry__.build()
    else:
        __graft_entry__.build()
        torch.cuda.set_device(local)
    import paper_0910_4497_gb300 as tb
    from paper_0910_4497_gb300 import binding as B

    cfg, pos, L, p = workload(args.workload)
    longrange = cfg.get("model") == "longrange"
    sampled = longrange or args.workload == "bridged6480"   # oracle on a bounded sample
    p["reorth_passes"] = args.reorth_passes
    p["reorth_every"] = args.reorth_every
    p["schedule"] = args.schedule
    grouped = args.group_m > 1
    if grouped:
        p["group_m"] = args.group_m
        p["max_union"] = args.max_union
    n = len(pos)
    cpu_base = None
    ref = None
    cpu_all = None
    lr_recs = None
    if rank == 0 and not args.no_cpu_baseline and sampled:
        # a full oracle evaluation of this cell takes minutes: a bounded sample
        t_atom, nu, lr_recs = oracle_target_sample(pos, L, p, k=4)
        cpu_base = {"value": 1.0 / t_atom, "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": f"the bond table of the {nu} atoms in the clusters of 4 targets "
                              f"and those targets' records (single process); value = 1 / "
                              f"(bond-table seconds per atom + record seconds per target)"}
    elif rank == 0 and not args.no_cpu_baseline:
        t_or, ref = time_oracle_full(pos, L, p)  # before any GPU work of this process
        cpu_base = {"value": n / t_or, "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": f"one full FP64 oracle force evaluation of the {n}-atom cell "
                              f"({t_or:.1f} s, single process)"}
        ncores = os.cpu_count() or 1
        if ncores > 1:
            import oracle
            t0 = time.perf_counter()
            oracle.force_evaluation(pos, L, p, workers=ncores, group_m=p.get("group_m", 1))
            t_all = time.perf_counter() - t0
            cpu_all = {"value": n / t_all, "unit": UNIT, "cores": ncores, "kind": "oracle",
                       "sample": f"the same evaluation with the targets spread over {ncores} "
                                 f"spawned worker processes ({t_all:.1f} s, pool start-up "
                                 f"included)"}
    dev = torch.device("cuda", local)
    system = tb.TBSystem(n, L, p, prec=args.prec, device=dev)
    B.tb_profile_enable(system.ctx, True)
    system.set_positions(pos)
    tune = None
    if args.prec != "fp64" and not grouped and not args.no_autotune:
        tune = system.autotune()
    system.capture()
    stream = torch.cuda.current_stream(dev)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    for _ in range(max(args.warmup, 3)):
        system.replay()
    torch.cuda.synchronize(dev)
    system.check()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    # ---- device-resident timed region
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    stage_ms = {k: [] for k in B.STAGES}
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.fill_(float(k))                       # evict L2 between steps
        ev[k][0].record(stream)
        system.replay()
        ev[k][1].record(stream)
        ev[k][1].synchronize()
        for name, v in B.tb_profile_read(system.ctx).items():
            stage_ms[name].append(v)
    barrier()
    clk = clocks.stop() if clocks else None
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, world, dev)
    system.check()
    value = job_throughput(n, world, args.steps, total_ms)
    accuracy = None
    if lr_recs is not None:
        e = system.energies.cpu().numpy()
        accuracy = {"vs": "FP64 CPU oracle spectral records of 4 sampled targets",
                    "moment_rel_err_max": sampled_moment_error(system, lr_recs, p["r"]),
                    "electron_count_err": float(abs(e[5] - 4 * n))}
    if ref is not None:
        import numpy as np
        F = system.F.cpu().numpy()
        e = system.energies.cpu().numpy()
        dF = np.abs(F - ref.F)
        accuracy = {"vs": "FP64 CPU oracle, same input",
                    "force_err_max_eV_per_A": float(dF.max()),
                    "force_err_rms_eV_per_A": float(np.sqrt(np.mean(dF ** 2))),
                    "band_energy_rel_err": float(abs(e[0] - ref.E_band) / abs(ref.E_band))}

    # ---- end to end through the public API with host buffers
    pin_pos = torch.as_tensor(pos, dtype=torch.float64).pin_memory()
    pin_F = torch.empty((n, 3), dtype=torch.float64).pin_memory()
    pin_E = torch.empty(8, dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.fill_(float(k))
        e0.record(stream)
        system.pos.copy_(pin_pos, non_blocking=True)
        system.replay()
        pin_F.copy_(system.F, non_blocking=True)
        pin_E.copy_(system.energies, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_value = job_throughput(n, world, args.steps, e2e_ms)

    if rank == 0:
        kry = [v for v in stage_ms["krylov"] if v > 0]
        kry_ms = statistics.mean(kry) if kry else None
        launches_per_step = B.tb_ctx_kernels_per_evaluation(system.ctx, n, L)
        mixed = args.prec != "fp64"
        # the mixed path runs the eigensolve inside the Krylov launch when the
        # library counts no separate eigensolver kernel
        if mixed and args.schedule != "auto":
            plan = args.schedule
        elif tune is not None:
            plan = tune["schedule"]
        elif mixed and not grouped and launches_per_step == list_launches(L, p["Rc"]) + 1 + 1 + 1 + 4:
            plan = "persistent"
        else:
            plan = "separate"
        persistent = plan in ("persistent", "persistent_largest_first")
        sweep_prec = "fp64" if not mixed else "mixed"
        sweep = (algorithmic_sweep_bytes_grouped(system, sweep_prec) if grouped
                 else algorithmic_sweep_bytes(system, sweep_prec))
        alg = sweep + (record_bytes(system, sweep_prec) if persistent else 0)
        peaks = {}
        pk = os.path.join(ROOT, "MEASURED_PEAKS.json")
        if os.path.exists(pk):
            peaks = json.load(open(pk))
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = alg / (kry_ms * 1e-3) / 1e9 if kry_ms else None
        kname = ("krylov_group_kernel (m-target block Lanczos on union clusters, one CTA "
                 "per group)" if grouped else
                 "kry_eig_kernel (block Lanczos targets then projected eigensolves from one "
                 "work queue)" if persistent else
                 "krylov_sk_kernel (one launch per cluster-size bucket; kernel_ms is the "
                 "Krylov stage, all launches)" if plan == "bucketed" else
                 "krylov_sk_kernel (block Lanczos on Slater-Koster records, one CTA per target)"
                 if mixed else
                 "krylov_kernel (FP64 block Lanczos, one CTA per target)")
        tkey = (args.prec if not mixed or grouped or longrange else
                "mixed" if persistent else "mixed_sweep_kernel")
        tr = kernel_traffic_record(tkey, "krylov_group_traffic.json" if grouped
                                   else "krylov_traffic_longrange.json" if longrange
                                   else "krylov_traffic.json", cfg["name"])
        traffic = tr.get("dram") if tr else None
        roof = {"bound": "hbm", "kernel": kname,
                "achieved": achieved, "peak": hbm, "unit": "GB/s",
                "peak_source": "measured" if "hbm_gbs" in peaks else "fallback",
                "frac": achieved / hbm if achieved else None,
                "traffic": traffic,
                "algorithmic_bytes": "sweep bytes of the scope table's definition (dense 4x4 "
                                     "bond blocks and the basis block, read and written, per "
                                     "sweep)" + (" plus the spectral records the launch "
                                                 "writes and reads back" if persistent else ""),
                "algorithmic_bytes_per_launch": alg, "kernel_ms": kry_ms,
                # measured DRAM use of the same launch (ncu record of this
                # workload) and its L2 traffic: the level that binds
                "dram_frac": (traffic / (kry_ms * 1e-3) / 1e9 / hbm
                              if traffic and kry_ms else None),
                "l2_bytes_per_launch": tr.get("l2") if tr else None,
                "l2_GBps": (tr["l2"] / (kry_ms * 1e-3) / 1e9
                            if tr and tr.get("l2") and kry_ms else None)}
        stages = {k: (statistics.mean([x for x in v if x >= 0]) if any(x >= 0 for x in v)
                      else None) for k, v in stage_ms.items()}
        extra = {}
        if mixed and not grouped and not args.no_fp64_compare:
            # the comparison the metric is named after: the plain FP64 path on
            # the same GPU, same cell, same Lanczos settings
            s64 = tb.TBSystem(n, L, p, prec="fp64", device=dev)
            B.tb_profile_enable(s64.ctx, True)
            s64.set_positions(pos)
            s64.capture()
            k64 = min(args.steps, 50)
            ms64, st64 = timed_leg(s64, k64, flush, stream, B)
            v64 = job_throughput(n, 1, k64, ms64 * k64)
            F64 = s64.F.cpu().numpy()
            s64.close()
            import numpy as np
            extra["fp64"] = {"value": v64, "unit": UNIT, "ms_per_step": ms64, "steps": k64,
                             "stage_ms": st64,
                             "mixed_vs_fp64_force_max_eV_per_A":
                                 float(np.abs(system.F.cpu().numpy() - F64).max())}
            extra["mixed_over_fp64"] = value / v64 / max(world, 1)
        if persistent:
            # the same sweeps as a separate launch, so that their own time and
            # roofline can be read apart from the eigensolves sharing the queue
            # (separate launches per size bucket with the autotuner's tiles: on
            # uniform clusters one bucket, i.e. the block-Lanczos kernel alone)
            sep = tb.TBSystem(n, L, dict(p, schedule="bucketed"), prec=args.prec, device=dev)
            B.tb_profile_enable(sep.ctx, True)
            sep.set_positions(pos)
            if not args.no_autotune:
                sep.autotune()
            sep.capture()
            ms_sep, st_sep = timed_leg(sep, min(args.steps, 100), flush, stream, B)
            sep.close()
            ksep = st_sep.get("krylov")
            a_sep = sweep / (ksep * 1e-3) / 1e9 if ksep else None
            trs = kernel_traffic_record("mixed_sweep_kernel", "krylov_traffic.json", cfg["name"])
            extra["roofline_sweeps"] = {
                "bound": "hbm", "kernel": "krylov_sk_kernel (separate launches per cluster-size "
                                          "bucket with the tuned tiles, same settings; kernel_ms "
                                          "is the Krylov stage)",
                "achieved": a_sep, "peak": hbm, "unit": "GB/s",
                "frac": a_sep / hbm if a_sep else None, "kernel_ms": ksep,
                "traffic": trs.get("dram") if trs else None,
                "l2_bytes_per_launch": trs.get("l2") if trs else None,
                "traffic_note": "ncu record of the default-tile separate launch",
                "algorithmic_bytes_per_launch": sweep,
                "step_ms_with_separate_launches": ms_sep}
        line = {
            "metric": METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": {"mixed": "f32+f64", "bf16": "bf16+f32+f64"}.get(args.prec, "f64"),
            "data": "synthetic",
            "config": config_dict(cfg, n, world),
            "run": {"precision": args.prec, "graph": "one CUDA graph per force evaluation",
                    "reorth_passes": args.reorth_passes, "reorth_every": args.reorth_every,
                    "schedule": plan,
                    **({"group_m": args.group_m, "max_union": args.max_union,
                        "form": "m-target union clusters (Eq. lanczos_blas3)"}
                       if grouped else {})},
            "e2e": {"value": e2e_value, "unit": UNIT, "h2d_bytes_per_step": n * 3 * 8,
                    "d2h_bytes_per_step": n * 3 * 8 + 8 * 8},
            "roofline": roof,
            "cpu_baseline": cpu_base,
            "cpu_baseline_all_cores": cpu_all,
            "clocks": clk,
            "gpu_launches": launches_per_step * args.steps,
            "stage_ms": stages,
            "accuracy": accuracy,
            "autotune": tune,
            **extra,
        }
        print(json.dumps(line), flush=True)
    system.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0

# ---------------------------------------------------------------- MD workload

MD_METRIC = "atom-steps/s (15360-atom C60 NVE MD, velocity Verlet, 1 GB300)"
MD_UNIT = "atom-steps/s"
MD_INDEX = 4


def md_workload():
    from synth import CONFIGS, fcc_c60_crystal, maxwell_boltzmann_velocities, workload_params
    from synth.configs import MASS_C_AMU
    cfg = CONFIGS[MD_INDEX]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"],
                                cfg["bridges"])
    vel = maxwell_boltzmann_velocities(len(pos), cfg["T_init"], MASS_C_AMU, cfg["seed"] + 1)
    p = workload_params(cfg, defl_tol=1e-9)
    return cfg, pos, vel, L, p


def oracle_md_sample(pos, L, p, n_targets):
    """Oracle per-target work (cluster H, block Lanczos, eigenpairs, density
    blocks) of n_targets evenly spaced targets; returns seconds per target."""
    from oracle.neighbors import neighbor_lists, cluster_lists
    from oracle.hamiltonian import BondTable
    from oracle.pipeline import target_record
    from oracle.density import rho_blocks
    hl = neighbor_lists(pos, L, p["rm"])
    cl = cluster_lists(pos, L, p["Rc"])
    bonds = BondTable(pos, L, hl, p)
    stride = max(1, len(pos) // n_targets)
    t0 = time.perf_counter()
    nt = 0
    for i in range(0, len(pos), stride):
        lam, S, P = target_record(bonds, cl[i], hl[i], p["r"], p["defl_tol"])
        rho_blocks(S, P, lam, 4.5, p["kT"])
        nt += 1
    return (time.perf_counter() - t0) / nt, nt


def md_trajectory(system, steps, flush, stream, record):
    """Replay `steps` MD graphs; per-step CUDA-event times and total energies."""
    import torch
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(steps)]
    etot = torch.zeros(steps, dtype=torch.float64, device=system.device)
    for k in range(steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        system.replay()
        ev[k][1].record(stream)
        etot[k:k + 1].copy_(system.energies[4:5] + system.energies[7:8])
        if record:
            ev[k][1].synchronize()
    torch.cuda.synchronize(system.device)
    return [a.elapsed_time(b) for a, b in ev], etot.cpu().numpy()


def run_md(args):
    import numpy as np
    import torch
    import __graft_entry__
    from synth.configs import MASS_C_AMU
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    if args.impl == "reference":
        if rank != 0:
            return 0
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        cfg, pos, vel, L, p = md_workload()
        t_tgt, nt = oracle_md_sample(pos, L, p, 64)
        value = 1.0 / t_tgt          # atom-steps/s: one target's work per atom-step
        line = {"metric": MD_METRIC, "value": value, "unit": MD_UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup,
                "ms_per_step": 1e3 * t_tgt * len(pos), "higher_is_better": True,
                "scaling": "weak", "vs_baseline": None, "dtype": "f64", "data": "synthetic",
                "impl": "reference",
                "config": {"workload": cfg["name"], "n_atoms": len(pos), "l2": "n/a (CPU)"},
                "cpu_baseline": {"value": value, "unit": MD_UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"per-target oracle work of {nt} evenly spaced "
                                           f"targets, scaled to one {len(pos)}-atom force "
                                           f"evaluation per MD step"},
                "e2e": {"value": value, "unit": MD_UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    if world > 1:
        import torch.distributed as dist
        if rank == 0:
            __graft_entry__.build()
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        dist.barrier()
        if rank != 0:
            __graft_entry__.build()
    else:
        __graft_entry__.build()
        torch.cuda.set_device(local)
    import paper_0910_4497_gb300 as tb

    cfg, pos, vel, L, p = md_workload()
    p["reorth_passes"] = args.reorth_passes
    p["reorth_every"] = args.reorth_every
    n = len(pos)
    dt = cfg["dt_fs"]
    cpu_base = None
    if rank == 0 and not args.no_cpu_baseline:
        t_tgt, nt = oracle_md_sample(pos, L, p, 64)
        cpu_base = {"value": 1.0 / t_tgt, "unit": MD_UNIT, "cores": 1, "kind": "oracle",
                    "sample": f"oracle per-target work (cluster H, block Lanczos, eigenpairs, "
                              f"density blocks) of {nt} evenly spaced targets, "
                              f"{t_tgt * nt:.1f} s, scaled to {n} targets per MD step"}
    dev = torch.device("cuda", local)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    tunes = {}

    def make(prec):
        s = tb.TBSystem(n, L, p, prec=prec, device=dev)
        tb.binding.tb_profile_enable(s.ctx, True)
        s.set_positions(pos)
        s.vel.copy_(torch.as_tensor(vel, dtype=torch.float64))
        if prec != "fp64" and not args.no_autotune:
            tunes[prec] = s.autotune()        # the launch plan of every step's graph
        s.evaluate()
        s.capture_md(dt, MASS_C_AMU)
        return s

    system = make(args.prec)
    for _ in range(max(args.warmup, 3)):
        system.replay()
    torch.cuda.synchronize(dev)
    system.check()
    state = [t.clone() for t in (system.pos, system.vel, system.F)]

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    barrier()
    step_ms, etot = md_trajectory(system, args.steps, flush, stream, True)
    barrier()
    stage_ms = tb.binding.tb_profile_read(system.ctx)     # the last step's stages
    clk = clocks.stop() if clocks else None
    system.check()
    total_ms = sum(step_ms)
    total_ms = max_over_ranks(total_ms, world, dev)
    value = job_throughput(n, world, args.steps, total_ms)
    pos_end = system.pos.clone()

    # ---- end to end: the state goes host -> device and back every step
    hp = [t.cpu().pin_memory() for t in state]
    hE = torch.empty(8, dtype=torch.float64).pin_memory()
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    e2e_ms = 0.0
    for k in range(args.steps):
        flush.fill_(float(k))
        e0.record(stream)
        for d, h in zip((system.pos, system.vel, system.F), hp):
            d.copy_(h, non_blocking=True)
        system.replay()
        for d, h in zip((system.pos, system.vel, system.F), hp):
            h.copy_(d, non_blocking=True)
        hE.copy_(system.energies, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    e2e_value = job_throughput(n, world, args.steps, e2e_ms)
    # kick-drift + one force evaluation + kick and its energy reduction
    launches_per_step = tb.binding.tb_ctx_kernels_per_evaluation(system.ctx, n, L) + 3
    system.close()

    # ---- the FP64 path over the same steps from the same state
    fp64 = None
    if rank == 0 and args.prec != "fp64" and not args.no_fp64_compare:
        s64 = tb.TBSystem(n, L, p, prec="fp64", device=dev)
        s64.set_positions(state[0])
        s64.vel.copy_(state[1])
        s64.evaluate()
        s64.capture_md(dt, MASS_C_AMU)
        ms64, etot64 = md_trajectory(s64, args.steps, flush, stream, True)
        s64.check()
        dpos = (s64.pos - pos_end + 0.5 * L).remainder(L) - 0.5 * L
        fp64 = {"atom_steps_per_s": n * args.steps / (sum(ms64) / 1e3),
                "ms_per_step": sum(ms64) / args.steps,
                "energy_drift_eV_per_atom": float((etot64[-1] - etot64[0]) / n),
                "max_position_diff_vs_mixed_A": float(dpos.abs().max().item())}
        s64.close()

    if rank == 0:
        line = {
            "metric": MD_METRIC, "value": value, "unit": MD_UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "n_atoms": n, "a": cfg["a"],
                       "ncell": cfg["ncell"], "Rc": cfg["Rc"], "krylov_r": cfg["r"],
                       "kT": cfg["kT"], "dt_fs": dt, "T_init_K": cfg["T_init"],
                       "precision": args.prec,
                       "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "graph": "one CUDA graph per MD step",
                       "reorth_passes": args.reorth_passes,
                       "reorth_every": args.reorth_every},
            "e2e": {"value": e2e_value, "unit": MD_UNIT, "h2d_bytes_per_step": 3 * n * 3 * 8,
                    "d2h_bytes_per_step": 3 * n * 3 * 8 + 8 * 8},
            "cpu_baseline": cpu_base,
            "clocks": clk,
            "gpu_launches": launches_per_step * args.steps,
            "stage_ms": stage_ms,
            "autotune": tunes.get(args.prec),
            "nve": {"energy_drift_eV_per_atom": float((etot[-1] - etot[0]) / n),
                    "energy_span_eV_per_atom": float((etot.max() - etot.min()) / n),
                    "fp64_path": fp64},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------- NPT workload

NPT_METRIC = ("atom-steps/s (15360-atom C60 NPT MD at 25 GPa and 500 K, velocity Verlet with "
              "weak coupling, 1 GB300)")


def intercage_bonds(system, cut=1.75):
    """Pairs of atoms of different C60 molecules (60 consecutive atoms each)
    closer than `cut`: the bonds of a polymerising crystal.  Rebuilds the
    system's own lists at its current positions and box first."""
    import numpy as np
    import torch
    system.neighbors()
    torch.cuda.synchronize()
    system.check()
    hl, _ = system.lists()
    x = system.pos.cpu().numpy()
    L = system.L
    count = 0
    for i, h in enumerate(hl):
        j = h[(h > i) & (h // 60 != i // 60)]
        if len(j):
            d = x[j] - x[i]
            d -= L * np.rint(d / L)
            count += int(np.sum(np.sum(d * d, axis=1) < cut * cut))
    return count


def run_npt(args):
    """Weak-coupling NPT steps of the 15360-atom cell at 25 GPa and 500 K."""
    import torch
    import __graft_entry__
    from synth import NPT, maxwell_boltzmann_velocities
    from synth.configs import MASS_C_AMU, GPA_PER_EV_A3
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    local = int(os.environ.get("LOCAL_RANK", "0"))
    cfg, pos, _, L, p = md_workload()
    vel = maxwell_boltzmann_velocities(len(pos), NPT["T0_K"], MASS_C_AMU, cfg["seed"] + 1)
    n = len(pos)
    dt = NPT["dt_fs"]
    P0 = NPT["P0_GPa"] / GPA_PER_EV_A3
    beta = GPA_PER_EV_A3 / NPT["B_GPa"]
    coupling = (NPT["T0_K"], P0, NPT["tau_T_fs"], NPT["tau_P_fs"], beta)
    wl = {"workload": NPT["name"], "n_atoms": n, "a": cfg["a"], "ncell": cfg["ncell"],
          "Rc": cfg["Rc"], "krylov_r": cfg["r"], "kT": cfg["kT"], "dt_fs": dt,
          "T0_K": NPT["T0_K"], "P0_GPa": NPT["P0_GPa"], "tau_T_fs": NPT["tau_T_fs"],
          "tau_P_fs": NPT["tau_P_fs"], "barostat_B_GPa": NPT["B_GPa"],
          "coupling": "Berendsen thermostat + isotropic Berendsen barostat"}
    if args.impl == "reference" and rank != 0:
        return 0
    if args.impl == "reference" or (rank == 0 and not args.no_cpu_baseline):
        t_tgt, nt = oracle_md_sample(pos, L, p, 64)
        cpu_base = {"value": 1.0 / t_tgt, "unit": MD_UNIT, "cores": 1, "kind": "oracle",
                    "sample": f"oracle per-target work of {nt} evenly spaced targets, scaled "
                              f"to one {n}-atom force evaluation per NPT step"}
    else:
        cpu_base = None
    if args.impl == "reference":
        v = cpu_base["value"]
        line = {"metric": NPT_METRIC, "value": v, "unit": MD_UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * n / v,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": dict(wl, l2="n/a (CPU)"), "cpu_baseline": cpu_base,
                "e2e": {"value": v, "unit": MD_UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    if world > 1:
        import torch.distributed as dist
        if rank == 0:
            __graft_entry__.build()
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        dist.barrier()
        if rank != 0:
            __graft_entry__.build()
    else:
        __graft_entry__.build()
        torch.cuda.set_device(local)
    import paper_0910_4497_gb300 as tb
    p["reorth_passes"] = args.reorth_passes
    p["reorth_every"] = args.reorth_every
    p["max_cluster"] = 256          # clusters grow as the box is compressed
    dev = torch.device("cuda", local)
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)
    s = tb.TBSystem(n, L, p, prec=args.prec, device=dev)
    s.set_positions(pos)
    s.vel.copy_(torch.as_tensor(vel, dtype=torch.float64))
    s.evaluate()
    # launch plan tuned once on the starting lists; targets whose clusters grow
    # as the box shrinks fall into the last size bucket (up to max_cluster)
    tune = s.autotune() if args.prec != "fp64" and not args.no_autotune else None
    bonds0 = intercage_bonds(s)
    for _ in range(max(args.warmup, 3)):
        s.npt_step(dt, MASS_C_AMU, *coupling)
    torch.cuda.synchronize(dev)
    s.check()

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    traj = []
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    barrier()
    for k in range(args.steps):
        flush.fill_(float(k))
        ev[k][0].record(stream)
        s.npt_step(dt, MASS_C_AMU, *coupling)       # ends with a read of the new box
        ev[k][1].record(stream)
        ev[k][1].synchronize()
        traj.append([s.L] + s.npt_state.cpu().tolist())
    barrier()
    clk = clocks.stop() if clocks else None
    s.check()
    step_ms = [a.elapsed_time(b) for a, b in ev]
    total_ms = max_over_ranks(sum(step_ms), world, dev)
    value = job_throughput(n, world, args.steps, total_ms)

    bonds1 = intercage_bonds(s)
    # ---- end to end: the state goes host -> device and back every step (at
    # most 20 steps: long trajectories are timed on the device only)
    e2e_steps = min(args.steps, 20)
    hp = [t.cpu().pin_memory() for t in (s.pos, s.vel, s.F)]
    hE = torch.empty(8, dtype=torch.float64).pin_memory()
    e2e_ms = 0.0
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    barrier()
    for k in range(e2e_steps):
        flush.fill_(float(k))
        e0.record(stream)
        for d, h in zip((s.pos, s.vel, s.F), hp):
            d.copy_(h, non_blocking=True)
        s.npt_step(dt, MASS_C_AMU, *coupling)
        for d, h in zip((s.pos, s.vel, s.F), hp):
            h.copy_(d, non_blocking=True)
        hE.copy_(s.energies, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    launches_per_step = tb.binding.tb_ctx_kernels_per_evaluation(s.ctx, n, L) + 5
    s.close()
    if rank == 0:
        tr = traj
        line = {
            "metric": NPT_METRIC, "value": value, "unit": MD_UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": dict(wl, precision=args.prec, l2="flushed between steps (256 MB write)",
                           parallelism=f"replicas x{world}" if world > 1 else "single GPU",
                           graph="none (the box changes every step; eager launches)",
                           reorth_passes=args.reorth_passes, reorth_every=args.reorth_every),
            "e2e": {"value": job_throughput(n, world, e2e_steps, e2e_ms), "unit": MD_UNIT,
                    "steps": e2e_steps,
                    "h2d_bytes_per_step": 3 * n * 3 * 8,
                    "d2h_bytes_per_step": 3 * n * 3 * 8 + 8 * 8 + 8},
            "cpu_baseline": cpu_base,
            "clocks": clk,
            "gpu_launches": launches_per_step * args.steps,
            "autotune": tune,
            "npt": {"L_A": [tr[0][0], tr[-1][0]], "T_K": [tr[0][1], tr[-1][1]],
                    "P_GPa": [tr[0][2] * GPA_PER_EV_A3, tr[-1][2] * GPA_PER_EV_A3],
                    "lambda_last": tr[-1][3], "mu_last": tr[-1][4],
                    "simulated_fs": (max(args.warmup, 3) + args.steps) * dt,
                    "intercage_bonds_lt_1p75A": [bonds0, bonds1],
                    "duration_3ps_s_at_this_rate": NPT["duration_ps"] * 1e3 / dt
                    * (total_ms / args.steps) / 1e3},
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------- exact local gradient

AG_METRIC = "atom force evals/s (exact local gradient at r = r_min, forward + backward, 1 GB300)"
AG_INDEX = 3


def ag_workload():
    from synth import CONFIGS, fcc_c60_crystal, workload_params
    cfg = CONFIGS[AG_INDEX]
    pos, L, _ = fcc_c60_crystal(cfg["ncell"], cfg["a"], cfg["jitter"], cfg["seed"],
                                cfg["bridges"])
    return cfg, pos, L, workload_params(cfg, defl_tol=1e-9)


def oracle_ag_sample(pos, L, p, n_targets):
    """Oracle per-target work of the exact local path (dense eigh of H_c, the
    Daleckii-Krein matrix and its bond contraction at a fixed mu) on evenly
    spaced targets; seconds per target."""
    import numpy as np
    from oracle.neighbors import neighbor_lists, cluster_lists
    from oracle.hamiltonian import BondTable
    from oracle import local_exact
    hl = neighbor_lists(pos, L, p["rm"])
    cl = cluster_lists(pos, L, p["Rc"])
    bonds = BondTable(pos, L, hl, p)
    F = np.zeros((len(pos), 3))
    stride = max(1, len(pos) // n_targets)
    t0 = time.perf_counter()
    nt = 0
    for i in range(0, len(pos), stride):
        lam, Z = local_exact.target_spectrum(bonds, cl[i])
        G = local_exact.target_gradient_matrix(lam, Z, 3.5, p["kT"])
        local_exact.target_force_terms(bonds, cl[i], G, F)
        nt += 1
    return (time.perf_counter() - t0) / nt, nt


def run_autograd(args):
    import numpy as np
    import torch
    import __graft_entry__
    from synth.c60 import wrap
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    cfg, pos, L, p = ag_workload()
    n = len(pos)
    if args.impl == "reference":
        if rank != 0:
            return 0
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        t_tgt, nt = oracle_ag_sample(pos, L, p, 16)
        value = 1.0 / t_tgt
        line = {"metric": AG_METRIC, "value": value, "unit": UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 * t_tgt * n,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": cfg["name"], "n_atoms": n, "l2": "n/a (CPU)"},
                "cpu_baseline": {"value": value, "unit": UNIT, "cores": 1, "kind": "oracle",
                                 "sample": f"dense eigh + Daleckii-Krein gradient of {nt} "
                                           f"evenly spaced targets, scaled to {n} targets"},
                "e2e": {"value": value, "unit": UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    if world > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        if rank == 0:
            __graft_entry__.build()
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        dist.barrier()
        if rank != 0:
            __graft_entry__.build()
    else:
        __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    dev = torch.device("cuda", torch.cuda.current_device())
    cpu_base = None
    if rank == 0 and not args.no_cpu_baseline:
        t_tgt, nt = oracle_ag_sample(pos, L, p, 16)
        cpu_base = {"value": 1.0 / t_tgt, "unit": UNIT, "cores": 1, "kind": "oracle",
                    "sample": f"dense eigh + Daleckii-Krein gradient of {nt} evenly spaced "
                              f"targets ({t_tgt * nt:.1f} s), scaled to {n} targets"}
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    def timed(system, steps, backward=True):
        f, b = [], []
        for k in range(steps):
            e = [torch.cuda.Event(enable_timing=True) for _ in range(3)]
            flush.fill_(float(k))
            e[0].record(stream)
            system.local_forward()
            e[1].record(stream)
            if backward:
                system.local_gradient()
            e[2].record(stream)
            e[2].synchronize()
            f.append(e[0].elapsed_time(e[1]))
            b.append(e[1].elapsed_time(e[2]))
        return f, b

    res = {}
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    for store in (True, False):
        s = tb.TBSystem(n, L, p, prec=args.prec, device=dev)
        s.reserve_local(store_basis=store)
        s.set_positions(pos)
        for _ in range(max(args.warmup, 3)):
            s.local_forward()
            s.local_gradient()
        barrier()
        f, b = timed(s, args.steps)
        barrier()
        s.check()
        res[store] = dict(fwd=f, bwd=b, F=s.F_loc.cpu().numpy(),
                          zbytes=(s.Z_loc.numel() * s.Z_loc.element_size()) if store else 0)
        if store:
            # end to end: positions from pinned host memory, forces and energies back
            hp = torch.as_tensor(pos, dtype=torch.float64).pin_memory()
            hF = torch.empty((n, 3), dtype=torch.float64).pin_memory()
            hE = torch.empty(8, dtype=torch.float64).pin_memory()
            e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
            barrier()
            e2e_ms = 0.0
            for k in range(args.steps):
                flush.fill_(float(k))
                e0.record(stream)
                s.pos.copy_(hp, non_blocking=True)
                s.local_forward()
                s.local_gradient()
                hF.copy_(s.F_loc, non_blocking=True)
                hE.copy_(s.energies_loc, non_blocking=True)
                e1.record(stream)
                e1.synchronize()
                e2e_ms += e0.elapsed_time(e1)
            res["e2e_ms"] = e2e_ms
        s.close()
    clk = clocks.stop() if clocks else None
    t_step = sum(a + b for a, b in zip(res[True]["fwd"], res[True]["bwd"]))
    t_step = max_over_ranks(t_step, world, dev)
    res["e2e_ms"] = max_over_ranks(res["e2e_ms"], world, dev)
    value = job_throughput(n, world, args.steps, t_step)
    check = None
    if rank == 0:
        # FP64 reference gradient and central differences of the FP64 energy
        s64 = tb.TBSystem(n, L, p, prec="fp64", device=dev)
        s64.reserve_local(store_basis=False)
        s64.set_positions(pos)
        s64.local_forward()
        s64.local_gradient()
        F64 = s64.F_loc.cpu().numpy()
        rng = np.random.default_rng(cfg["seed"])
        h = 1e-4
        fd_err, crossings, errs = 0.0, [], []
        c_off0, c_idx0 = s64.c_off.clone(), s64.c_idx.clone()
        for q in rng.choice(3 * n, size=args.fd_coords, replace=False):
            atom, k = divmod(int(q), 3)
            ev = []
            same = True
            for sgn in (1.0, -1.0):
                x = pos.copy()
                x[atom, k] += sgn * h
                s64.set_positions(wrap(x, L))
                s64.local_forward()
                ev.append(s64.energies_loc[4].item())
                same = same and torch.equal(s64.c_off, c_off0) and torch.equal(s64.c_idx, c_idx0)
            e = abs(-(ev[0] - ev[1]) / (2 * h) - F64[atom, k])
            errs.append(e)
            # the truncated local energy jumps where an atom crosses a cluster's
            # cutoff sphere: a difference across such a crossing is not a derivative
            if same:
                fd_err = max(fd_err, e)
            else:
                crossings.append({"atom": atom, "axis": k, "err_eV_per_A": e})
        s64.check()
        s64.close()
        check = {"fd_coords": args.fd_coords, "fd_h_A": h,
                 "fd_vs_fp64_gradient_max_eV_per_A": fd_err,
                 "fd_vs_fp64_gradient_median_eV_per_A": float(np.median(errs)),
                 "fd_coords_crossing_a_cluster_cutoff": crossings,
                 "force_vs_fp64_path_max_eV_per_A": float(np.abs(res[True]["F"] - F64).max()),
                 "stored_equals_recomputed": bool(np.array_equal(res[True]["F"],
                                                                 res[False]["F"]))}
        mean = statistics.mean
        line = {
            "metric": AG_METRIC, "value": value, "unit": UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": t_step / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": cfg["name"], "n_atoms": n, "a": cfg["a"], "Rc": cfg["Rc"],
                       "krylov_r": "r_min (dense cluster eigenproblem)", "kT": cfg["kT"],
                       "precision": args.prec, "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "step": "forward (spectra, mu, energies) + stored-basis backward"},
            "e2e": {"value": job_throughput(n, world, args.steps, res["e2e_ms"]), "unit": UNIT,
                    "h2d_bytes_per_step": n * 3 * 8, "d2h_bytes_per_step": n * 3 * 8 + 64},
            "roofline": None,
            "cpu_baseline": cpu_base,
            "clocks": clk,
            # lists + assembly + spectra + mu + energies + reduction + gradient + gather
            "gpu_launches": (list_launches(L, p["Rc"]) + 7) * args.steps,
            "backward": {"forward_ms": mean(res[True]["fwd"]),
                         "stored_basis_ms": mean(res[True]["bwd"]),
                         "recomputed_basis_ms": mean(res[False]["bwd"]),
                         "stored_basis_bytes": res[True]["zbytes"],
                         "recomputed_basis_bytes": 0},
            "check": check,
        }
        print(json.dumps(line), flush=True)
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


# ---------------------------------------------------------------- diamond equation of state

EOS_METRIC = "pressure evaluations/s (4x4x4 diamond supercell, 512 atoms, 1 GB300)"
EOS_UNIT = "pressure evaluations/s"
GPA = 160.21766208


def eos_params(a, r=None):
    from synth import DIAMOND_EOS, TB_CONSTANTS
    d = DIAMOND_EOS
    p = dict(TB_CONSTANTS)
    p.update(kT=d["kT"], Rc=d["Rc_over_a"] * a, r=d["r"] if r is None else r,
             max_hnbr=d["max_hnbr"], max_cluster=d["max_cluster"], n_electrons_per_atom=4.0,
             defl_tol=1e-9)
    return p


def oracle_pressure(a, ncell):
    """One full oracle force evaluation plus virial of the perfect diamond cell."""
    import oracle
    from oracle import virial
    from synth import diamond_cell
    pos, L = diamond_cell(ncell, a)
    p = eos_params(a)
    t0 = time.perf_counter()
    res = oracle.force_evaluation(pos, L, p)
    W = virial.evaluation_virial(res, p)
    dt = time.perf_counter() - t0
    return dt, virial.pressure(W, L), res.E_total / len(pos)


def birch_murnaghan(V, E):
    """Third-order Birch-Murnaghan fit: E = sum_k c_k V^{-2k/3}, k = 0..3."""
    import numpy as np
    x = V ** (-2.0 / 3.0)
    c = np.polyfit(x, E, 3)
    xs = np.roots(np.polyder(c))
    xs = xs[np.isreal(xs)].real
    xs = xs[(xs > x.min() * 0.8) & (xs < x.max() * 1.2)]
    if len(xs) == 0:
        return None
    x0 = xs[np.argmin(np.polyval(c, xs))]
    V0 = x0 ** (-1.5)
    # B = V d2E/dV2 at V0, with x = V^{-2/3}: dE/dV = E'(x) (-2/3) V^{-5/3}
    d1, d2 = np.polyval(np.polyder(c), x0), np.polyval(np.polyder(c, 2), x0)
    B0 = V0 * (d2 * (4.0 / 9.0) * V0 ** (-10.0 / 3.0) + d1 * (10.0 / 9.0) * V0 ** (-8.0 / 3.0))
    def P_of(V):
        xv = V ** (-2.0 / 3.0)
        return np.polyval(np.polyder(c), xv) * (2.0 / 3.0) * V ** (-5.0 / 3.0)
    return dict(V0_A3_per_atom=float(V0), a0_A=float((8 * V0) ** (1 / 3)),
                B0_GPa=float(B0 * GPA), P_fit=P_of)


def run_eos(args):
    import numpy as np
    import torch
    import __graft_entry__
    from synth import DIAMOND_EOS, diamond_cell
    d = DIAMOND_EOS
    rank = int(os.environ.get("RANK", "0"))
    world = int(os.environ.get("WORLD_SIZE", "1"))
    a_ref = 3.55
    if args.impl == "reference":
        if rank != 0:
            return 0
        os.environ.setdefault("OMP_NUM_THREADS", "1")
        os.environ.setdefault("OPENBLAS_NUM_THREADS", "1")
        ts = []
        for k in range(args.warmup + args.steps):
            dt, _, _ = oracle_pressure(d["a_list"][k % len(d["a_list"])], d["ncell"])
            if k >= args.warmup:
                ts.append(dt)
        value = len(ts) / sum(ts)
        line = {"metric": EOS_METRIC, "value": value, "unit": EOS_UNIT, "n_gpus": args.gpus,
                "steps": args.steps, "warmup": args.warmup, "ms_per_step": 1e3 / value,
                "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
                "dtype": "f64", "data": "synthetic", "impl": "reference",
                "config": {"workload": d["name"], "n_atoms": 512, "l2": "n/a (CPU)"},
                "cpu_baseline": {"value": value, "unit": EOS_UNIT, "cores": 1, "kind": "oracle",
                                 "sample": "full oracle force evaluation + virial of the 512-atom "
                                           "cell per step, lattice constants cycled"},
                "e2e": {"value": value, "unit": EOS_UNIT, "h2d_bytes_per_step": 0,
                        "d2h_bytes_per_step": 0}}
        print(json.dumps(line), flush=True)
        return 0
    if world > 1:
        import torch.distributed as dist
        local = int(os.environ.get("LOCAL_RANK", "0"))
        if rank == 0:
            __graft_entry__.build()
        torch.cuda.set_device(local)
        dist.init_process_group("nccl")
        dist.barrier()
        if rank != 0:
            __graft_entry__.build()
    else:
        __graft_entry__.build()
    import paper_0910_4497_gb300 as tb
    from paper_0910_4497_gb300 import binding as B
    dev = torch.device("cuda", torch.cuda.current_device())
    cpu_base, ref = None, None
    if rank == 0 and not args.no_cpu_baseline:
        t_or, P_or, e_or = oracle_pressure(a_ref, d["ncell"])
        cpu_base = {"value": 1.0 / t_or, "unit": EOS_UNIT, "cores": 1, "kind": "oracle",
                    "sample": f"one full oracle force evaluation + virial of the 512-atom cell "
                              f"at a = {a_ref} A ({t_or:.1f} s, single process)"}
        ref = (P_or, e_or)
    systems = []
    for a in d["a_list"]:
        pos, L = diamond_cell(d["ncell"], a)
        s = tb.TBSystem(len(pos), L, eos_params(a), prec=args.prec, device=dev)
        B.tb_profile_enable(s.ctx, True)
        s.set_positions(pos)
        s.capture(with_virial=True)
        systems.append((a, pos, L, s))
    n = len(systems[0][1])
    flush = torch.empty(256 * 1024 * 1024 // 4, dtype=torch.float32, device=dev)
    stream = torch.cuda.current_stream(dev)

    def barrier():
        if world > 1:
            torch.distributed.barrier()
        torch.cuda.synchronize(dev)

    for k in range(max(args.warmup, 3)):
        systems[k % len(systems)][3].replay()
    barrier()
    clocks = ClockSampler(torch.cuda.current_device()) if rank == 0 else None
    ev = [(torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True))
          for _ in range(args.steps)]
    kry = []
    for k in range(args.steps):
        s = systems[k % len(systems)][3]
        flush.fill_(float(k))
        ev[k][0].record(stream)
        s.replay()
        ev[k][1].record(stream)
        ev[k][1].synchronize()
        kry.append(B.tb_profile_read(s.ctx)["krylov"])
    barrier()
    clk = clocks.stop() if clocks else None
    total_ms = sum(a.elapsed_time(b) for a, b in ev)
    total_ms = max_over_ranks(total_ms, world, dev)
    value = job_throughput(1, world, args.steps, total_ms)
    # end to end: positions in, energies and pressure out
    e0, e1 = torch.cuda.Event(enable_timing=True), torch.cuda.Event(enable_timing=True)
    hp = [torch.as_tensor(x[1], dtype=torch.float64).pin_memory() for x in systems]
    hout = torch.empty(8 + 9 + 1, dtype=torch.float64).pin_memory()
    e2e_ms = 0.0
    barrier()
    for k in range(args.steps):
        q = k % len(systems)
        s = systems[q][3]
        flush.fill_(float(k))
        e0.record(stream)
        s.pos.copy_(hp[q], non_blocking=True)
        s.replay()
        hout[:8].copy_(s.energies, non_blocking=True)
        hout[8:17].copy_(s.W, non_blocking=True)
        hout[17:].copy_(s.pressure, non_blocking=True)
        e1.record(stream)
        e1.synchronize()
        e2e_ms += e0.elapsed_time(e1)
    e2e_ms = max_over_ranks(e2e_ms, world, dev)
    # equation of state and its convergence (untimed)
    table = []
    for a, pos, L, s in systems:
        s.replay()
        torch.cuda.synchronize(dev)
        s.check()
        e = s.energies.cpu().numpy()
        table.append(dict(a_A=a, V_A3_per_atom=L ** 3 / n, E_eV_per_atom=float(e[4] / n),
                          P_GPa=float(s.pressure.item() * GPA),
                          max_abs_F=float(s.F.abs().max().item())))
    conv = []
    if rank == 0:
        for a, _, _, _ in systems:
            row = {"a_A": a}
            for tag, ncell, r in (("r12", d["ncell"], d["r_check"]), ("8x8x8", d["ncell_big"], None)):
                pos, L = diamond_cell(ncell, a)
                s2 = tb.TBSystem(len(pos), L, eos_params(a, r), prec=args.prec, device=dev)
                s2.set_positions(pos)
                s2.evaluate(with_virial=True)
                torch.cuda.synchronize(dev)
                s2.check()
                row[f"P_GPa_{tag}"] = float(s2.pressure.item() * GPA)
                row[f"E_eV_per_atom_{tag}"] = float(s2.energies[4].item() / len(pos))
                s2.close()
            conv.append(row)
    V = np.array([t["V_A3_per_atom"] for t in table])
    E = np.array([t["E_eV_per_atom"] for t in table])
    fit = birch_murnaghan(V, E)
    if fit is not None:
        Pf = fit.pop("P_fit")
        for t in table:
            t["P_GPa_from_fit"] = float(Pf(t["V_A3_per_atom"]) * GPA)
    if rank == 0:
        alg = algorithmic_sweep_bytes(systems[0][3], args.prec)
        kms = [v for v in kry if v > 0]
        kry_ms = statistics.mean(kms) if kms else None
        peaks = json.load(open(os.path.join(ROOT, "MEASURED_PEAKS.json"))) if os.path.exists(
            os.path.join(ROOT, "MEASURED_PEAKS.json")) else {}
        hbm = peaks.get("hbm_gbs", 6800.0)
        achieved = alg / (kry_ms * 1e-3) / 1e9 if kry_ms else None
        acc = None
        if ref is not None:
            sr = systems[[x[0] for x in systems].index(a_ref)][3]
            acc = {"vs": f"FP64 CPU oracle at a = {a_ref} A",
                   "pressure_err_GPa": float(abs(sr.pressure.item() - ref[0]) * GPA),
                   "energy_err_eV_per_atom": float(abs(sr.energies[4].item() / n - ref[1]))}
        line = {
            "metric": EOS_METRIC, "value": value, "unit": EOS_UNIT, "n_gpus": world,
            "steps": args.steps, "warmup": args.warmup, "ms_per_step": total_ms / args.steps,
            "higher_is_better": True, "scaling": "weak", "vs_baseline": None,
            "dtype": "f32+f64" if args.prec == "mixed" else "f64", "data": "synthetic",
            "config": {"workload": d["name"], "n_atoms": n, "a_A": d["a_list"],
                       "Rc": "1.26 a (71 atoms per cluster)", "krylov_r": d["r"], "kT": d["kT"],
                       "precision": args.prec, "l2": "flushed between steps (256 MB write)",
                       "parallelism": f"replicas x{world}" if world > 1 else "single GPU",
                       "graph": "one CUDA graph per pressure evaluation"},
            "e2e": {"value": job_throughput(1, world, args.steps, e2e_ms), "unit": EOS_UNIT,
                    "h2d_bytes_per_step": n * 3 * 8, "d2h_bytes_per_step": 18 * 8},
            "roofline": {"bound": "hbm", "kernel": "krylov_kernel", "achieved": achieved,
                         "peak": hbm, "unit": "GB/s", "frac": achieved / hbm if achieved else None,
                         "traffic": None, "algorithmic_bytes_per_launch": alg,
                         "kernel_ms": kry_ms},
            "cpu_baseline": cpu_base,
            "clocks": clk,
            # one force evaluation + the virial per step
            "gpu_launches": (B.tb_ctx_kernels_per_evaluation(systems[0][3].ctx, n, systems[0][2])
                             + 1) * args.steps,
            "paper_context": {"seconds_gpu_8800gtx_xu": 55.65, "seconds_cpu_elses_xu": 29.19,
                              "note": "time to compute the pressure of the 4x4x4 supercell; the "
                                      "number of evaluations inside is not stated"},
            "eos": table,
            "birch_murnaghan": fit,
            "convergence": conv,
            "accuracy": acc,
        }
        print(json.dumps(line), flush=True)
    for _, _, _, s in systems:
        s.close()
    if world > 1:
        torch.distributed.destroy_process_group()
    return 0


def main():
    args = parse()
    if args.workload == "autograd1920":
        return run_autograd(args)
    if args.workload == "diamond_eos":
        return run_eos(args)
    if args.workload == "md15360":
        return run_md(args)
    if args.workload == "npt15360":
        return run_npt(args)
    if args.impl == "reference":
        return run_reference(args)
    return run_ours(args)


if __name__ == "__main__":
    sys.exit(main())
