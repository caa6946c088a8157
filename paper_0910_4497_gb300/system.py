"""Device buffers for one periodic cell and the call sequence of one force
evaluation through the C ABI (a1..a10), optionally captured as a CUDA graph.

PyTorch is used only to own device memory and streams; every step of the
evaluation runs in libtb.so.
"""
import torch

from . import binding as B


class TBSystem:
    """One cell of n atoms in a cubic box of side L.

    params: dict with the model constants (Es, Ep, Vss, Vsp, Vpps, Vppp, r0, n, nc,
    rc, phi0, d0, m, mc, dc, r1, rm), kT, Rc, r, and optionally max_hnbr,
    max_cluster, defl_tol, reorth_passes, mu_tol, mu_max_iter.
    prec: "fp64", "mixed" or "bf16" (mixed with BF16 H.V sweeps).
    """

    def __init__(self, n, L, params, prec="fp64", device="cuda"):
        self.n, self.L = int(n), float(L)
        self.prec = prec
        self.params = dict(params)
        self.tp = B.make_params(self.params, prec)
        self.NT = 4 * self.tp.r
        self.device = torch.device(device)
        with torch.cuda.device(self.device):
            self.ctx = B.tb_ctx_create(self.tp)
            B.tb_ctx_reserve(self.ctx, self.n)
        n, NT, mh, mc = self.n, self.NT, self.tp.max_hnbr, self.tp.max_cluster
        kw = dict(device=self.device)
        i32, f64, f32 = torch.int32, torch.float64, torch.float32
        self.pos = torch.zeros((n, 3), dtype=f64, **kw)
        self.h_off = torch.zeros(n + 1, dtype=i32, **kw)
        self.h_idx = torch.zeros(n * mh, dtype=i32, **kw)
        self.c_off = torch.zeros(n + 1, dtype=i32, **kw)
        self.c_idx = torch.zeros(n * mc, dtype=i32, **kw)
        self.Hblk = torch.zeros(n * mh * 16, dtype=f64, **kw)
        self.dHblk = torch.zeros(n * mh * 48, dtype=f64, **kw)
        # Slater-Koster records (s(r), l) of the bonds for the mixed and BF16 sweeps
        self.Hsk = torch.zeros(n * mh * 4, dtype=f32, **kw) if self.tp.prec != B.TB_PREC_FP64 else None
        self.lam = torch.zeros(n * NT, dtype=f64, **kw)
        self.S = torch.zeros(n * 4 * NT, dtype=f64, **kw)
        self.P = torch.zeros((n + n * mh) * 4 * NT, dtype=f64, **kw)
        self.kdim = torch.zeros(n, dtype=i32, **kw)
        self.mu = torch.full((1,), float("nan"), dtype=f64, **kw)
        self.ncount = torch.zeros(1, dtype=f64, **kw)
        self.F = torch.zeros((n, 3), dtype=f64, **kw)
        self.vel = torch.zeros((n, 3), dtype=f64, **kw)
        self.energies = torch.zeros(8, dtype=f64, **kw)
        self.W = torch.zeros(9, dtype=f64, **kw)
        self.pressure = torch.zeros(1, dtype=f64, **kw)
        self.L_dev = torch.zeros(1, dtype=f64, **kw)        # box after an NPT scaling
        self.npt_state = torch.zeros(4, dtype=f64, **kw)    # T (K), P (eV/A^3), lambda, mu
        # m-target form: groups of group_m targets (tb_group_atoms)
        self.group_m = self.tp.group_m
        self.n_groups = (n + self.group_m - 1) // self.group_m
        self.g_off = torch.zeros(self.n_groups + 1, dtype=i32, **kw)
        self.g_idx = torch.zeros(n, dtype=i32, **kw)
        self.graph = None

    # -- the five stages of one force evaluation
    def neighbors(self, stream=None):
        B.tb_build_neighbors(self.ctx, self.n, self.pos, self.L, self.h_off, self.h_idx,
                             self.c_off, self.c_idx, stream)

    def assemble(self, stream=None):
        B.tb_assemble_H(self.ctx, self.n, self.pos, self.L, self.h_off, self.h_idx,
                        self.Hblk, self.dHblk, self.Hsk, stream)

    def krylov(self, stream=None):
        """Block Krylov runs and projected eigensolve of every target; with
        group_m > 1 the m-target form on the groups in g_off / g_idx."""
        if self.group_m > 1:
            B.tb_krylov_density_grouped(self.ctx, self.n, self.n_groups, self.g_off, self.g_idx,
                                        self.c_off, self.c_idx, self.h_off, self.h_idx,
                                        self.Hblk, self.Hsk, self.lam, self.S, self.P,
                                        self.kdim, stream)
            return
        B.tb_krylov_density(self.ctx, self.n, self.c_off, self.c_idx, self.h_off,
                            self.h_idx, self.Hblk, self.Hsk, self.lam, self.S, self.P,
                            self.kdim, stream)

    def autotune(self, stream=None):
        """Lists and bond records of the positions in self.pos, then the
        library's autotuner on them (mixed / BF16 path, before capture());
        returns its report (cluster-size histogram, plan times, bucket tiles)."""
        self.neighbors(stream)
        self.assemble(stream)
        return B.tb_autotune(self.ctx, self.n, self.c_off, self.c_idx, self.h_off, self.h_idx,
                             self.Hblk, self.Hsk, self.lam, self.S, self.P, self.kdim, stream)

    def group(self, stream=None):
        """Spatial groups of group_m targets of the positions in self.pos."""
        B.tb_group_atoms(self.ctx, self.n, self.pos, self.L, self.g_off, self.g_idx, stream)

    def find_mu(self, stream=None, warm_start=True):
        B.tb_find_mu(self.ctx, self.n, self.lam, self.S, self.kdim, 4.0 * self.n,
                     self.mu if warm_start else None, self.mu, self.ncount, stream)

    def forces(self, stream=None):
        B.tb_forces(self.ctx, self.n, self.pos, self.L, self.h_off, self.h_idx, self.dHblk,
                    self.lam, self.S, self.P, self.kdim, self.mu, self.F, self.energies,
                    stream)

    def evaluate(self, stream=None, warm_start=False, with_virial=False):
        """One full force evaluation (lists to forces) of the positions in self.pos;
        with_virial adds the virial W (3x3, eV) and static pressure (eV/A^3)."""
        self.neighbors(stream)
        if self.group_m > 1:
            self.group(stream)
        self.assemble(stream)
        self.krylov(stream)
        self.find_mu(stream, warm_start=warm_start)
        self.forces(stream)
        if with_virial:
            self.virial(stream)

    def virial(self, stream=None):
        """Virial and static pressure from the last forces() call."""
        B.tb_virial(self.ctx, self.n, self.pos, self.L, self.h_off, self.h_idx, self.W,
                    self.pressure, stream)

    def md_step(self, dt_fs, mass_amu, stream=None):
        B.tb_md_step(self.ctx, self.n, self.pos, self.vel, self.F, self.L, dt_fs, mass_amu,
                     self.energies, stream)

    def npt_step(self, dt_fs, mass_amu, T0, P0, tau_T_fs, tau_P_fs, beta, stream=None):
        """One velocity-Verlet step at the current box, its virial, and the
        weak-coupling NPT scaling.  Updates self.L from the device (one
        device-to-host read, which waits for the step); the step's T, P and
        scale factors are left in self.npt_state."""
        self.md_step(dt_fs, mass_amu, stream)
        B.tb_virial(self.ctx, self.n, self.pos, self.L, None, None, self.W, self.pressure,
                    stream)
        B.tb_npt_berendsen(self.ctx, self.n, self.pos, self.vel, self.L, self.W, self.energies,
                           T0, P0, dt_fs, tau_T_fs, tau_P_fs, beta, self.L_dev,
                           self.npt_state, stream)
        if stream is not None:
            stream.synchronize()
        self.L = float(self.L_dev.item())

    # -- checkpoint / restart of a trajectory
    def checkpoint(self, path, step, seed):
        """Write pos, vel, F, the box, the step count and the seed (host copy)."""
        from . import checkpoint as ck
        ck.save(path, self.pos.cpu().numpy(), self.vel.cpu().numpy(), self.F.cpu().numpy(),
                self.L, step, seed, params=self.params, prec=self.prec)

    def restore(self, path):
        """Load a checkpoint written by checkpoint() into this system (same n);
        returns (step, seed).  Recapture a step graph afterwards if the box
        changed."""
        from . import checkpoint as ck
        st = ck.load(path)
        if st["pos"].shape[0] != self.n:
            raise ValueError(f"checkpoint holds {st['pos'].shape[0]} atoms, system {self.n}")
        for t, k in ((self.pos, "pos"), (self.vel, "vel"), (self.F, "F")):
            t.copy_(torch.as_tensor(st[k]))
        self.L = st["L"]
        return st["step"], st["seed"]

    # -- exact local free energy and its gradient at r = r_min
    def reserve_local(self, store_basis=False):
        """Dense workspace and buffers of the exact local path; with store_basis
        the forward keeps every target's eigenvectors for the backward
        (n * (4 max_cluster)^2 elements), else the backward recomputes them."""
        B.tb_ctx_reserve_local(self.ctx, self.n)
        n, ND = self.n, 4 * self.tp.max_cluster
        kw = dict(device=self.device)
        f64 = torch.float64
        self.ND = ND
        self.lam_loc = torch.zeros(n * ND, dtype=f64, **kw)
        self.S_loc = torch.zeros(n * 4 * ND, dtype=f64, **kw)
        self.kdim_loc = torch.zeros(n, dtype=torch.int32, **kw)
        self.mu_loc = torch.zeros(1, dtype=f64, **kw)
        self.energies_loc = torch.zeros(8, dtype=f64, **kw)
        self.F_loc = torch.zeros((n, 3), dtype=f64, **kw)
        zt = f64 if self.tp.prec == B.TB_PREC_FP64 else torch.float32
        self.Z_loc = torch.zeros(n * ND * ND, dtype=zt, **kw) if store_basis else None
        self.local_version = 0

    def local_forward(self, stream=None):
        """Lists, bond blocks, dense spectra of every cluster, mu and energies
        (energies_loc[4] = A_loc + E_rep) of the positions in self.pos."""
        self.neighbors(stream)
        self.assemble(stream)
        B.tb_local_forward(self.ctx, self.n, self.pos, self.L, self.c_off, self.c_idx,
                           self.h_off, self.h_idx, self.Hblk, self.lam_loc, self.S_loc,
                           self.kdim_loc, self.Z_loc, self.mu_loc, self.energies_loc, stream)
        self.local_version += 1

    def local_gradient(self, stream=None):
        """F_loc = -d(A_loc + E_rep)/dR at the last local_forward's state."""
        B.tb_local_gradient(self.ctx, self.n, self.pos, self.L, self.c_off, self.c_idx,
                            self.h_off, self.h_idx, self.Hblk, self.dHblk, self.lam_loc,
                            self.S_loc, self.Z_loc, self.mu_loc, self.F_loc, stream)

    # -- CUDA graph of one evaluation
    def capture(self, with_virial=False):
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        with torch.cuda.stream(s):
            for _ in range(2):
                self.evaluate(s, with_virial=with_virial)
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        self.check()
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.evaluate(with_virial=with_virial)
        self.graph = g
        return g

    def capture_md(self, dt_fs, mass_amu):
        """CUDA graph of one velocity-Verlet step (self.F must hold the force at
        self.pos); replay() then advances the trajectory by one step."""
        s = torch.cuda.Stream(device=self.device)
        s.wait_stream(torch.cuda.current_stream(self.device))
        saved = [t.clone() for t in (self.pos, self.vel, self.F, self.mu)]
        with torch.cuda.stream(s):
            self.md_step(dt_fs, mass_amu, s)
        torch.cuda.current_stream(self.device).wait_stream(s)
        torch.cuda.synchronize(self.device)
        self.check()
        for t, v in zip((self.pos, self.vel, self.F, self.mu), saved):
            t.copy_(v)
        g = torch.cuda.CUDAGraph()
        with torch.cuda.graph(g):
            self.md_step(dt_fs, mass_amu)
        self.graph = g
        return g

    def replay(self):
        self.graph.replay()

    def set_positions(self, pos):
        self.pos.copy_(torch.as_tensor(pos, dtype=torch.float64), non_blocking=True)

    def check(self, stream=None):
        code, info = B.tb_get_status(self.ctx, stream)
        if code != B.TB_OK:
            raise B.TBError("device status", code, info)

    def status(self, stream=None):
        return B.tb_get_status(self.ctx, stream)

    # -- views for comparisons
    def lists(self):
        ho = self.h_off.cpu().numpy()
        hi = self.h_idx.cpu().numpy()
        co = self.c_off.cpu().numpy()
        ci = self.c_idx.cpu().numpy()
        return ([hi[ho[i]:ho[i + 1]] for i in range(self.n)],
                [ci[co[i]:co[i + 1]] for i in range(self.n)])

    def close(self):
        if getattr(self, "ctx", None) is not None:
            B.tb_ctx_destroy(self.ctx)
            self.ctx = None

    def __del__(self):
        try:
            self.close()
        except Exception:
            pass
