// C ABI entry points: argument checks, context and workspace management, and
// the stream-ordered launch sequence of each call.  Kernels live in the other
// translation units.
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <cmath>
#include <nvtx3/nvToolsExt.h>
#include "tb_internal.cuh"

// Tracing: every stream-ordered entry point opens an NVTX range named after
// itself for the duration of the host call (a profiler or tracing tool shows
// them on the host timeline; without one attached they cost a few ns).
namespace {
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
};
}  // namespace
#define TB_NVTX(name) NvtxRange tb_nvtx_range_(name)

size_t krylov_basis_bytes_global(const tb_ctx* c);

namespace {

bool finite_pos(double x) { return x == x && x < 1e300 && x > -1e300; }

tb_status check_params(const tb_params& p) {
  if (!(p.kT > 0.0) || !(p.Rc >= p.rm) || !(p.rm > p.r1) || !(p.r1 > 0.0)) return TB_ERR_INVALID_ARG;
  if (!(p.r0 > 0.0) || !(p.rc > 0.0) || !(p.dc > 0.0) || !(p.d0 > 0.0)) return TB_ERR_INVALID_ARG;
  if (p.r < 1 || p.r > tbk::MAX_R) return TB_ERR_INVALID_ARG;
  if (p.prec != TB_PREC_FP64 && p.prec != TB_PREC_MIXED && p.prec != TB_PREC_BF16)
    return TB_ERR_INVALID_ARG;
  if (p.prec == TB_PREC_BF16 && p.group_m > 1) return TB_ERR_INVALID_ARG;
  if (p.max_hnbr < 1 || p.max_hnbr > tbk::MAX_HNBR) return TB_ERR_INVALID_ARG;
  if (p.max_cluster < 1 || p.max_cluster > tbk::MAX_CLUSTER) return TB_ERR_INVALID_ARG;
  if (p.reorth_passes < 1 || p.reorth_passes > 2) return TB_ERR_INVALID_ARG;
  if (p.reorth_every < 1) return TB_ERR_INVALID_ARG;
  if (p.group_m < 1 || p.group_m > 4) return TB_ERR_INVALID_ARG;
  if (p.max_union < 0 || p.max_union > tbk::MAX_CLUSTER) return TB_ERR_INVALID_ARG;
  if (p.mu_max_iter < 1 || !(p.mu_tol > 0.0) || !(p.defl_tol >= 0.0)) return TB_ERR_INVALID_ARG;
  if (p.timeout_cycles <= 0) return TB_ERR_INVALID_ARG;
  if (p.schedule < TB_SCHED_AUTO || p.schedule > TB_SCHED_BUCKETED) return TB_ERR_INVALID_ARG;
  if (!finite_pos(p.Es) || !finite_pos(p.Ep)) return TB_ERR_INVALID_ARG;
  return TB_OK;
}

size_t align256(size_t x) { return (x + 255) & ~size_t(255); }

struct Carver {
  unsigned char* base;
  size_t off = 0;
  template <typename T>
  T* take(size_t count) {
    T* p = base ? reinterpret_cast<T*>(base + off) : nullptr;
    off += align256(sizeof(T) * count);
    return p;
  }
};

// Lays out every workspace sub-buffer; with base == nullptr only sizes them.
size_t carve(tb_ctx* c, int n, unsigned char* base) {
  const tb_params& p = c->p;
  const size_t NT = 4 * (size_t)p.r;
  const size_t hcap = (size_t)n * p.max_hnbr;
  const size_t rows = (size_t)n + hcap;   // row blocks of Y, P, rho
  const size_t tv = p.prec == TB_PREC_FP64 ? sizeof(double) : sizeof(float);
  Carver k{base};
  c->scan_h = k.take<int>(n + 1);
  c->scan_c = k.take<int>(n + 1);
  const size_t ncell = neighbor_cell_capacity(n);
  c->cell_cnt = k.take<int>(ncell);
  c->cell_off = k.take<int>(ncell + 1);
  c->cell_atoms = k.take<int>(n);
  c->atom_cell = k.take<int>(n);
  c->pad_h = k.take<int>(hcap);
  c->pad_c = k.take<int>((size_t)n * p.max_cluster);
  c->T = k.take<double>((size_t)n * tc_doubles(p.r));
  c->Y = k.take<unsigned char>(rows * 4 * NT * tv);
  c->colmask = k.take<unsigned long long>(n);
  c->Zf = k.take<float>((size_t)n * NT * NT);
  c->lamf = k.take<float>((size_t)n * NT);
  c->Vg = k.take<unsigned char>(krylov_basis_bytes_global(c));
  c->lent = k.take<int2>(p.prec == TB_PREC_FP64
                             ? (size_t)c->kry_grid * p.max_cluster * p.max_hnbr : 0);
  c->bref = k.take<int2>(krylov_overflow_records(c));
  c->ke_work = k.take<int>((size_t)n + 1);
  c->tgt_order = k.take<int>(n);
  c->tgt_boff = k.take<int>(tb_plan::MAX_BINS + 1);
  c->grp_V = k.take<unsigned char>(krylov_group_basis_bytes(c));
  c->grp_lent = k.take<int2>((size_t)c->grp_grid * c->grp_max_union * p.max_hnbr);
  c->grp_cnt = k.take<int>(n);
  c->grp_off = k.take<int>(n + 1);
  c->grp_idx = k.take<int>(n);
  c->mu_part = k.take<double>(2 * 16 * (size_t)(c->mu_grid > 0 ? c->mu_grid : 1));
  c->bar = k.take<unsigned>(4);
  c->mu_state = k.take<double>(4);
  c->rho = k.take<double>(rows * 16 > (size_t)n * 2 ? rows * 16 : (size_t)n * 2);
  c->per_target = k.take<double>((size_t)n * 5 + 4 * ((size_t)n / 64 + 1));   // + energy partials
  c->bondf = k.take<double>(hcap * 4);
  c->h_off = k.take<int>(n + 1);
  c->h_idx = k.take<int>(hcap);
  c->c_off = k.take<int>(n + 1);
  c->c_idx = k.take<int>((size_t)n * p.max_cluster);
  c->Hblk = k.take<double>(hcap * 16);
  c->dHblk = k.take<double>(hcap * 48);
  c->Hsk = k.take<float>(hcap * 4);
  c->lambda = k.take<double>((size_t)n * NT);
  c->S = k.take<double>((size_t)n * 4 * NT);
  c->P = k.take<double>(rows * 4 * NT);
  c->kdim = k.take<int>(n);
  c->mu = k.take<double>(1);
  c->ncount = k.take<double>(1);
  return k.off;
}

tb_status ready(tb_ctx* c, int n) {
  if (!c) return TB_ERR_INVALID_ARG;
  if (n < 0) return TB_ERR_INVALID_ARG;
  if (n > c->reserved_n || !c->ws) return TB_ERR_NOT_RESERVED;
  return TB_OK;
}

}  // namespace

tb_status prof_mark(tb_ctx* c, int stage, bool end, cudaStream_t s) {
  if (!c->profiling) return TB_OK;
  cudaEvent_t ev = c->prof_ev[2 * stage + (end ? 1 : 0)];
  cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
  TB_CUDA_TRY(cudaStreamIsCapturing(s, &cs));
  if (cs == cudaStreamCaptureStatusActive) {
    TB_CUDA_TRY(cudaEventRecordWithFlags(ev, s, cudaEventRecordExternal));
  } else {
    TB_CUDA_TRY(cudaEventRecord(ev, s));
  }
  if (end) c->prof_ran[stage] = true;
  return TB_OK;
}

#define TB_STAGE(c, stage, s, call)                                  \
  do {                                                               \
    tb_status st_ = prof_mark((c), (stage), false, (s));             \
    if (st_ != TB_OK) return st_;                                    \
    st_ = (call);                                                    \
    if (st_ != TB_OK) return st_;                                    \
    st_ = prof_mark((c), (stage), true, (s));                        \
    if (st_ != TB_OK) return st_;                                    \
  } while (0)

extern "C" {

tb_status tb_params_default(tb_params* p) {
  if (!p) return TB_ERR_INVALID_ARG;
  std::memset(p, 0, sizeof(*p));
  p->kT = 0.1;
  p->Rc = 5.0;
  p->r1 = 2.45;
  p->rm = 2.6;
  p->defl_tol = 1e-9;
  p->mu_tol = 1e-12;
  p->r = 8;
  p->prec = TB_PREC_FP64;
  p->max_hnbr = 32;
  p->max_cluster = 128;
  p->reorth_passes = 2;
  p->reorth_every = 1;
  p->group_m = 1;
  p->max_union = 0;
  p->mu_max_iter = 100;
  p->timeout_cycles = 4000000000LL;
  return TB_OK;
}

tb_status tb_ctx_create(tb_ctx** out, const tb_params* p) {
  if (!out || !p) return TB_ERR_INVALID_ARG;
  *out = nullptr;
  tb_status st = check_params(*p);
  if (st != TB_OK) return st;
  tb_ctx* c = new (std::nothrow) tb_ctx();
  if (!c) return TB_ERR_NOMEM;
  c->p = *p;
  if (cudaGetDevice(&c->device) != cudaSuccess ||
      cudaDeviceGetAttribute(&c->num_sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess) {
    delete c;
    return TB_ERR_CUDA;
  }
  if ((st = krylov_configure(c)) != TB_OK || (st = eig_configure(c)) != TB_OK ||
      (st = mu_configure(c)) != TB_OK ||
      (p->group_m > 1 && (st = krylov_group_configure(c)) != TB_OK)) {
    delete c;
    return st;
  }
  if (cudaMalloc(&c->d_status, 2 * sizeof(int)) != cudaSuccess) {
    delete c;
    return TB_ERR_NOMEM;
  }
  if (cudaMemset(c->d_status, 0, 2 * sizeof(int)) != cudaSuccess) {
    cudaFree(c->d_status);
    delete c;
    return TB_ERR_CUDA;
  }
  *out = c;
  return TB_OK;
}

tb_status tb_ctx_destroy(tb_ctx* c) {
  if (!c) return TB_ERR_INVALID_ARG;
  cudaDeviceSynchronize();
  if (c->ws) cudaFree(c->ws);
  if (c->loc_ws) cudaFree(c->loc_ws);
  if (c->d_status) cudaFree(c->d_status);
  for (int q = 0; q < 14; ++q)
    if (c->prof_ev[q]) cudaEventDestroy(c->prof_ev[q]);
  delete c;
  return TB_OK;
}

tb_status tb_ctx_reserve(tb_ctx* c, int n_atoms) {
  if (!c || n_atoms < 0) return TB_ERR_INVALID_ARG;
  if (n_atoms <= c->reserved_n && c->ws) return TB_OK;
  const size_t bytes = carve(c, n_atoms, nullptr);
  if (c->ws) {
    cudaDeviceSynchronize();
    cudaFree(c->ws);
    c->ws = nullptr;
    c->reserved_n = 0;
    c->ws_bytes = 0;
  }
  unsigned char* ws = nullptr;
  if (cudaMalloc(&ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    return TB_ERR_NOMEM;
  }
  carve(c, n_atoms, ws);
  c->ws = ws;
  c->ws_bytes = bytes;
  c->reserved_n = n_atoms;
  TB_CUDA_TRY(cudaMemset(ws, 0, bytes));
  TB_CUDA_TRY(cudaMemset(c->mu, 0xff, sizeof(double)));   // NaN: no previous mu
  TB_CUDA_TRY(cudaDeviceSynchronize());
  return TB_OK;
}

tb_status tb_ctx_workspace_bytes(const tb_ctx* c, size_t* bytes) {
  if (!c || !bytes) return TB_ERR_INVALID_ARG;
  *bytes = c->ws_bytes;
  return TB_OK;
}

tb_status tb_get_status(tb_ctx* c, int* code, int* info, void* stream) {
  if (!c || !code) return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  int h[2] = {0, 0};
  TB_CUDA_TRY(cudaMemcpyAsync(h, c->d_status, sizeof(h), cudaMemcpyDeviceToHost, s));
  TB_CUDA_TRY(cudaMemsetAsync(c->d_status, 0, sizeof(h), s));
  TB_CUDA_TRY(cudaStreamSynchronize(s));
  *code = h[0];
  if (info) *info = h[1];
  return TB_OK;
}

tb_status tb_build_neighbors(tb_ctx* c, int n, const double* pos, double L, int* h_off,
                             int* h_idx, int* c_off, int* c_idx, void* stream) {
  TB_NVTX("tb_build_neighbors");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (n == 0) return TB_OK;
  if (!pos || !h_off || !h_idx || !c_off || !c_idx || !(L > 0.0) || !finite_pos(L))
    return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TB_STAGE(c, 0, s, launch_neighbors(c, n, pos, L, h_off, h_idx, c_off, c_idx, s));
  return TB_OK;
}

tb_status tb_assemble_H(tb_ctx* c, int n, const double* pos, double L, const int* h_off,
                        const int* h_idx, double* Hblk, double* dHblk, float* Hsk,
                        void* stream) {
  TB_NVTX("tb_assemble_H");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (n == 0) return TB_OK;
  if (!pos || !h_off || !h_idx || !Hblk || !dHblk || !(L > 0.0)) return TB_ERR_INVALID_ARG;
  if (c->p.prec != TB_PREC_FP64 && !Hsk) return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TB_STAGE(c, 1, s, launch_assemble(c, n, pos, L, h_off, h_idx, Hblk, dHblk, Hsk, s));
  return TB_OK;
}

tb_status tb_krylov_density(tb_ctx* c, int n, const int* c_off, const int* c_idx,
                            const int* h_off, const int* h_idx, const double* Hblk,
                            const float* Hsk, double* lambda, double* S, double* P,
                            int* kdim, void* stream) {
  TB_NVTX("tb_krylov_density");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (n == 0) return TB_OK;
  if (!c_off || !c_idx || !h_off || !h_idx || !lambda || !S || !P || !kdim)
    return TB_ERR_INVALID_ARG;
  if (c->p.prec == TB_PREC_FP64 && !Hblk) return TB_ERR_INVALID_ARG;
  if (c->p.prec != TB_PREC_FP64 && !Hsk) return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TB_STAGE(c, 2, s, launch_krylov(c, n, c_off, c_idx, h_off, h_idx, Hblk, Hsk, lambda, S,
                                  P, kdim, s));
  TB_STAGE(c, 3, s, launch_eig(c, n, h_off, lambda, S, P, kdim, s));
  return TB_OK;
}

tb_status tb_group_atoms(tb_ctx* c, int n, const double* pos, double L, int* g_off, int* g_idx,
                         void* stream) {
  TB_NVTX("tb_group_atoms");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (n == 0) return TB_OK;
  if (!pos || !g_off || !g_idx || !(L > 0.0)) return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TB_STAGE(c, 6, s, launch_group_atoms(c, n, pos, L, g_off, g_idx, s));
  return TB_OK;
}

tb_status tb_krylov_density_grouped(tb_ctx* c, int n, int n_groups, const int* g_off,
                                    const int* g_idx, const int* c_off, const int* c_idx,
                                    const int* h_off, const int* h_idx, const double* Hblk,
                                    const float* Hsk, double* lambda, double* S, double* P,
                                    int* kdim, void* stream) {
  TB_NVTX("tb_krylov_density_grouped");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (c->p.group_m < 2 || c->grp_grid <= 0) return TB_ERR_INVALID_ARG;
  if (n == 0) return TB_OK;
  if (n_groups < 1 || n_groups > n) return TB_ERR_INVALID_ARG;
  if (!g_off || !g_idx || !c_off || !c_idx || !h_off || !h_idx || !lambda || !S || !P || !kdim)
    return TB_ERR_INVALID_ARG;
  if (c->p.prec == TB_PREC_FP64 && !Hblk) return TB_ERR_INVALID_ARG;
  if (c->p.prec != TB_PREC_FP64 && !Hsk) return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TB_STAGE(c, 2, s, launch_krylov_grouped(c, n, n_groups, g_off, g_idx, c_off, c_idx, h_off,
                                          h_idx, Hblk, Hsk, s));
  TB_STAGE(c, 3, s, launch_eig(c, n, h_off, lambda, S, P, kdim, s));
  return TB_OK;
}

tb_status tb_find_mu(tb_ctx* c, int n, const double* lambda, const double* S, const int* kdim,
                     double n_electrons, const double* mu_guess, double* mu, double* n_count,
                     void* stream) {
  TB_NVTX("tb_find_mu");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (!lambda || !S || !kdim || !mu || n <= 0 || !(n_electrons > 0.0)) return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TB_STAGE(c, 4, s, launch_mu(c, n, lambda, S, n_electrons, mu_guess, mu, n_count, s));
  return TB_OK;
}

tb_status tb_forces(tb_ctx* c, int n, const double* pos, double L, const int* h_off,
                    const int* h_idx, const double* dHblk, const double* lambda,
                    const double* S, const double* P, const int* kdim, const double* mu,
                    double* F, double* energies, void* stream) {
  TB_NVTX("tb_forces");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (n == 0) return TB_OK;
  if (!pos || !h_off || !h_idx || !dHblk || !lambda || !S || !P || !kdim || !mu || !F ||
      !energies || !(L > 0.0))
    return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  TB_STAGE(c, 5, s, launch_forces(c, n, pos, L, h_off, h_idx, dHblk, lambda, S, P, kdim, mu,
                                  F, energies, s));
  return TB_OK;
}

tb_status tb_md_step(tb_ctx* c, int n, double* pos, double* vel, double* F, double L,
                     double dt_fs, double mass_amu, double* energies, void* stream) {
  TB_NVTX("tb_md_step");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (n == 0) return TB_OK;
  if (!pos || !vel || !F || !energies || !(L > 0.0) || !(mass_amu > 0.0) || !(dt_fs > 0.0))
    return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  if ((st = launch_md_kick_drift(c, n, pos, vel, F, L, dt_fs, mass_amu, s)) != TB_OK) return st;
  const bool grouped = c->p.group_m > 1;
  TB_STAGE(c, 0, s, launch_neighbors(c, n, pos, L, c->h_off, c->h_idx, c->c_off, c->c_idx, s));
  if (grouped) TB_STAGE(c, 6, s, launch_group_atoms(c, n, pos, L, c->grp_off, c->grp_idx, s));
  TB_STAGE(c, 1, s, launch_assemble(c, n, pos, L, c->h_off, c->h_idx, c->Hblk, c->dHblk,
                                    c->p.prec != TB_PREC_FP64 ? c->Hsk : nullptr, s));
  if (grouped) {
    const int G = (n + c->p.group_m - 1) / c->p.group_m;
    TB_STAGE(c, 2, s, launch_krylov_grouped(c, n, G, c->grp_off, c->grp_idx, c->c_off,
                                            c->c_idx, c->h_off, c->h_idx, c->Hblk, c->Hsk, s));
  } else {
    TB_STAGE(c, 2, s, launch_krylov(c, n, c->c_off, c->c_idx, c->h_off, c->h_idx, c->Hblk,
                                    c->Hsk, c->lambda, c->S, c->P, c->kdim, s));
  }
  TB_STAGE(c, 3, s, launch_eig(c, n, c->h_off, c->lambda, c->S, c->P, c->kdim, s));
  TB_STAGE(c, 4, s, launch_mu(c, n, c->lambda, c->S, 4.0 * n, c->mu, c->mu, c->ncount, s));
  TB_STAGE(c, 5, s, launch_forces(c, n, pos, L, c->h_off, c->h_idx, c->dHblk, c->lambda, c->S,
                                  c->P, c->kdim, c->mu, F, energies, s));
  return launch_md_kick(c, n, vel, F, dt_fs, mass_amu, energies, s);
}

tb_status tb_virial(tb_ctx* c, int n, const double* pos, double L, const int* h_off,
                    const int* h_idx, double* W, double* pressure, void* stream) {
  TB_NVTX("tb_virial");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (!h_off && !h_idx) {      // the context's own lists, as left by tb_md_step
    h_off = c->h_off;
    h_idx = c->h_idx;
  }
  if (!pos || !h_off || !h_idx || !W || !(L > 0.0)) return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return launch_virial(c, n, pos, L, h_off, h_idx, W, pressure, s);
}

tb_status tb_npt_berendsen(tb_ctx* c, int n, double* pos, double* vel, double L,
                           const double* W, const double* energies, double T0, double P0,
                           double dt_fs, double tau_T_fs, double tau_P_fs, double beta,
                           double* L_new, double* state, void* stream) {
  TB_NVTX("tb_npt_berendsen");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (!pos || !vel || !W || !energies || !L_new || !state || !(L > 0.0) || !(T0 >= 0.0) ||
      !(dt_fs > 0.0) || !(tau_T_fs > dt_fs) || !(tau_P_fs > dt_fs) || !(beta > 0.0) ||
      !std::isfinite(P0))
    return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return launch_npt_berendsen(c, n, pos, vel, L, W, energies, T0, P0, dt_fs, tau_T_fs, tau_P_fs,
                              beta, L_new, state, s);
}

tb_status tb_ctx_reserve_local(tb_ctx* c, int n_atoms) {
  if (!c || n_atoms < 0) return TB_ERR_INVALID_ARG;
  if (n_atoms <= c->loc_reserved_n && c->loc_ws) return TB_OK;
  tb_status st = local_configure(c);
  if (st != TB_OK) return st;
  const size_t bytes = local_workspace_bytes(c, n_atoms);
  if (c->loc_ws) {
    cudaDeviceSynchronize();
    cudaFree(c->loc_ws);
    c->loc_ws = nullptr;
    c->loc_reserved_n = 0;
  }
  unsigned char* ws = nullptr;
  if (cudaMalloc(&ws, bytes) != cudaSuccess) {
    cudaGetLastError();
    return TB_ERR_NOMEM;
  }
  local_carve(c, n_atoms, ws);
  c->loc_ws = ws;
  c->loc_reserved_n = n_atoms;
  TB_CUDA_TRY(cudaMemset(ws, 0, bytes));
  TB_CUDA_TRY(cudaDeviceSynchronize());
  return TB_OK;
}

tb_status tb_local_forward(tb_ctx* c, int n, const double* pos, double L, const int* c_off,
                           const int* c_idx, const int* h_off, const int* h_idx,
                           const double* Hblk, double* lambda, double* S, int* kdim,
                           void* Zstore, double* mu, double* energies, void* stream) {
  TB_NVTX("tb_local_forward");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (n > c->loc_reserved_n || !c->loc_ws) return TB_ERR_NOT_RESERVED;
  if (n == 0) return TB_OK;
  if (!pos || !c_off || !c_idx || !h_off || !h_idx || !Hblk || !lambda || !S || !kdim || !mu ||
      !energies || !(L > 0.0))
    return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return launch_local_forward(c, n, pos, L, c_off, c_idx, h_off, h_idx, Hblk, lambda, S, kdim,
                              Zstore, mu, energies, s);
}

tb_status tb_local_gradient(tb_ctx* c, int n, const double* pos, double L, const int* c_off,
                            const int* c_idx, const int* h_off, const int* h_idx,
                            const double* Hblk, const double* dHblk, const double* lambda,
                            const double* S, const void* Zstore, const double* mu, double* F,
                            void* stream) {
  TB_NVTX("tb_local_gradient");
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (n > c->loc_reserved_n || !c->loc_ws) return TB_ERR_NOT_RESERVED;
  if (n == 0) return TB_OK;
  if (!pos || !c_off || !c_idx || !h_off || !h_idx || !Hblk || !dHblk || !lambda || !S || !mu ||
      !F || !(L > 0.0))
    return TB_ERR_INVALID_ARG;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  return launch_local_gradient(c, n, pos, L, c_off, c_idx, h_off, h_idx, Hblk, dHblk, lambda, S,
                               Zstore, mu, F, s);
}

tb_status tb_autotune(tb_ctx* c, int n, const int* c_off, const int* c_idx, const int* h_off,
                      const int* h_idx, const double* Hblk, const float* Hsk, double* lambda,
                      double* S, double* P, int* kdim, tb_tune_report* report, void* stream) {
  TB_NVTX("tb_autotune");
  (void)Hblk;
  tb_status st = ready(c, n);
  if (st != TB_OK) return st;
  if (!c_off || !c_idx || !h_off || !h_idx || !Hsk || !lambda || !S || !P || !kdim)
    return TB_ERR_INVALID_ARG;
  return krylov_autotune(c, n, c_off, c_idx, h_off, h_idx, Hsk, lambda, S, P, kdim, report,
                         static_cast<cudaStream_t>(stream));
}

tb_status tb_ctx_kernels_per_evaluation(const tb_ctx* c, int n, double L, int* count) {
  if (!c || !count || n < 0 || !(L > 0.0)) return TB_ERR_INVALID_ARG;
  if (n > c->reserved_n || !c->ws) return TB_ERR_NOT_RESERVED;
  const bool mixed = c->p.prec != TB_PREC_FP64;
  int k = neighbor_kernel_count(c, L) + 1;            // lists, assembly
  int eig = mixed ? 1 : 2;                             // group eigensolver (+ FP64 refinement)
  if (c->p.group_m > 1) {
    k += 2 + 1;                                        // grouping; grouped block Lanczos
  } else {
    k += krylov_kernel_count(c, n);                    // block Lanczos (+ size bins)
    if (krylov_eig_persistent(c, n)) eig = 0;          // eigensolve inside the Krylov launch
  }
  *count = k + eig + 1 + 3;                            // mu; rho, bond forces, sums and energies
  return TB_OK;
}

tb_status tb_profile_enable(tb_ctx* c, int enable) {
  if (!c) return TB_ERR_INVALID_ARG;
  if (enable) {
    for (int q = 0; q < 14; ++q)
      if (!c->prof_ev[q]) TB_CUDA_TRY(cudaEventCreate(&c->prof_ev[q]));
  }
  c->profiling = enable != 0;
  return TB_OK;
}

tb_status tb_profile_read(tb_ctx* c, float* ms) {
  if (!c || !ms) return TB_ERR_INVALID_ARG;
  for (int q = 0; q < 7; ++q) {
    ms[q] = -1.f;
    if (c->prof_ev[2 * q] && c->prof_ran[q]) {
      float t = -1.f;
      if (cudaEventElapsedTime(&t, c->prof_ev[2 * q], c->prof_ev[2 * q + 1]) == cudaSuccess)
        ms[q] = t;
      else
        cudaGetLastError();
    }
  }
  return TB_OK;
}

const char* tb_version(void) { return "tb-gb300 0.1.0 (sm_103a)"; }

}  // extern "C"
