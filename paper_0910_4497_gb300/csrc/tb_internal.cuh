// Internal declarations shared by the library's translation units.
#pragma once
#include <cuda_runtime.h>
#include <stdint.h>
#include "tb.h"

#define TB_CUDA_TRY(call)                                  \
  do {                                                     \
    cudaError_t e_ = (call);                               \
    if (e_ != cudaSuccess) return TB_ERR_CUDA;             \
  } while (0)

// Block-tridiagonal T of one target, stored compactly: 2r - 1 blocks of 16
// doubles, block 2k = A_k (row-major), block 2k+1 = B_k with
// T[4(k+1)+j][4k+c] = T[4k+c][4(k+1)+j] = B_k[j][c].
__host__ __device__ __forceinline__ size_t tc_doubles(int r) { return (size_t)(2 * r - 1) * 16; }
// Index of T[x][y] in the compact form, or -1 outside the block band.
__host__ __device__ __forceinline__ int tc_index(int x, int y) {
  const int kx = x >> 2, ky = y >> 2, jx = x & 3, jy = y & 3;
  if (kx == ky) return 32 * kx + 4 * jx + jy;
  if (kx == ky + 1) return 32 * ky + 16 + 4 * jx + jy;
  if (ky == kx + 1) return 32 * kx + 16 + 4 * jy + jx;
  return -1;
}

namespace tb_plan {
constexpr int MAX_BUCKETS = TB_TUNE_MAX_BUCKETS;
constexpr int MAX_BINS = TB_TUNE_BINS;
constexpr int BIN = 8;                // atoms per size bin
}

// Tile of one launch of the mixed-path block-Lanczos kernel.
struct tb_sk_cfg {
  int mc = 0;                         // cluster capacity of the basis blocks
  int ecap = 0;                       // Slater-Koster records in shared memory
  int minb = 4;                       // CTAs per SM the register budget allows
  int grid = 0;                       // CTAs of the launch
  size_t smem = 0;
};

namespace tbk {

constexpr int MAX_R = 16;           // Krylov block order cap -> NT <= 64
constexpr int MAX_NT = 4 * MAX_R;
constexpr int MAX_HNBR = 256;       // Hamiltonian list capacity (long-range hoppings: ~170 at 7 A)
constexpr int MAX_CLUSTER = 1024;

// Device status word: [0] = first tb_status code, [1] = qualifying info.
__device__ __forceinline__ void set_status(int* st, int code, int info) {
  if (atomicCAS(st, 0, code) == 0) atomicExch(st + 1, info);
}

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Fixed-order block reduction of M values per thread (M <= 16).  Every thread
// passes its partials; on return out[0..M) (shared) holds the totals.  Uses
// red[nwarps*M] shared scratch.  Contains two __syncthreads().
template <typename T, int M>
__device__ __forceinline__ void block_sum(T (&v)[M], T* red, T* out) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
#pragma unroll
  for (int q = 0; q < M; ++q) v[q] = warp_sum(v[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < M; ++q) red[warp * M + q] = v[q];
  }
  __syncthreads();
  if (threadIdx.x < M) {
    T s = 0;
    for (int w = 0; w < nw; ++w) s += red[w * M + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// Sum 16 per-lane values over the warp with a butterfly that halves the
// number of live values at every step (16 shuffles instead of 80).  On return
// lanes with (lane & 1) == 0 hold the total of value index (lane >> 1).
template <typename T>
__device__ __forceinline__ T warp_reduce16(const T (&v)[16], int lane) {
  T a8[8];
  const bool h16 = lane & 16;
#pragma unroll
  for (int j = 0; j < 8; ++j) {
    const T send = h16 ? v[j] : v[8 + j];
    const T keep = h16 ? v[8 + j] : v[j];
    a8[j] = keep + __shfl_xor_sync(0xffffffffu, send, 16);
  }
  T a4[4];
  const bool h8 = lane & 8;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const T send = h8 ? a8[j] : a8[4 + j];
    const T keep = h8 ? a8[4 + j] : a8[j];
    a4[j] = keep + __shfl_xor_sync(0xffffffffu, send, 8);
  }
  T a2[2];
  const bool h4 = lane & 4;
#pragma unroll
  for (int j = 0; j < 2; ++j) {
    const T send = h4 ? a4[j] : a4[2 + j];
    const T keep = h4 ? a4[2 + j] : a4[j];
    a2[j] = keep + __shfl_xor_sync(0xffffffffu, send, 4);
  }
  const bool h2 = lane & 2;
  const T a1 = (h2 ? a2[1] : a2[0]) + __shfl_xor_sync(0xffffffffu, h2 ? a2[0] : a2[1], 2);
  return a1 + __shfl_xor_sync(0xffffffffu, a1, 1);
}

// Block reduction of M <= 16 values per thread through the butterfly above:
// same contract as block_sum (red needs nwarps*16 entries).
template <typename T, int M>
__device__ __forceinline__ void block_sum16(const T (&v)[M], T* red, T* out) {
  static_assert(M <= 16, "at most 16 values");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int nw = blockDim.x >> 5;
  T p[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) p[q] = q < M ? v[q] : T(0);
  const T t = warp_reduce16(p, lane);
  if ((lane & 1) == 0 && (lane >> 1) < M) red[warp * 16 + (lane >> 1)] = t;
  __syncthreads();
  if (threadIdx.x < M) {
    T s = 0;
    for (int w = 0; w < nw; ++w) s += red[w * 16 + threadIdx.x];
    out[threadIdx.x] = s;
  }
  __syncthreads();
}

// The same reduction with the totals formed by every thread (NW warps): no
// second barrier and no broadcast; the partial sums are added in warp order,
// as in block_sum16, so every thread gets the bits block_sum16 would give.
// `red` must not be written again before every thread has read it.
template <typename T, int M, int NW>
__device__ __forceinline__ void block_sum_all(const T (&v)[M], T* red, T (&out)[M]) {
  static_assert(M <= 16, "at most 16 values");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  T p[16];
#pragma unroll
  for (int q = 0; q < 16; ++q) p[q] = q < M ? v[q] : T(0);
  const T t = warp_reduce16(p, lane);
  if ((lane & 1) == 0 && (lane >> 1) < M) red[warp * 16 + (lane >> 1)] = t;
  __syncthreads();
#pragma unroll
  for (int q = 0; q < M; ++q) {
    T s = 0;
#pragma unroll
    for (int w = 0; w < NW; ++w) s += red[w * 16 + q];
    out[q] = s;
  }
}

}  // namespace tbk

struct tb_ctx {
  tb_params p;
  int device = 0;
  int num_sms = 0;
  int* d_status = nullptr;           // 2 ints
  // workspace
  int reserved_n = 0;
  size_t ws_bytes = 0;
  unsigned char* ws = nullptr;
  // sub-buffers inside ws
  int* scan_h = nullptr;             // n+1 counts (H lists)
  int* scan_c = nullptr;             // n+1 counts (clusters)
  int* cell_cnt = nullptr;           // neighbour cells: counts (cell capacity)
  int* cell_off = nullptr;           // offsets (cell capacity + 1)
  int* cell_atoms = nullptr;         // n atoms binned by cell
  int* atom_cell = nullptr;          // n cell ids
  int* pad_h = nullptr;              // n * max_hnbr padded Hamiltonian lists
  int* pad_c = nullptr;              // n * max_cluster padded clusters
  double* T = nullptr;               // n * tc_doubles(r): compact block-tridiagonal T
  void* Y = nullptr;                 // n*(1+max_hnbr)*4*NT  (TV precision)
  unsigned long long* colmask = nullptr;  // n
  float* Zf = nullptr;               // n * NT * NT
  float* lamf = nullptr;             // n * NT
  void* Vg = nullptr;                // kry_grid * Dmax * NT (TV) when the basis is global
  int2* lent = nullptr;              // kry_grid * max_cluster * max_hnbr (slot, bond), FP64 path
  int2* bref = nullptr;              // mixed path: per-CTA overflow of the local
                                     //   sparsity (bond index, neighbour offset)
  double* mu_part = nullptr;         // mu_grid * 4
  unsigned int* bar = nullptr;       // barrier counter
  double* mu_state = nullptr;        // 4 doubles
  double* rho = nullptr;             // n*(1+max_hnbr)*16
  double* per_target = nullptr;      // n * 5
  double* bondf = nullptr;           // n*max_hnbr*4: per-bond force and half repulsion
  double* dscratch = nullptr;        // eig refinement scratch
  // MD-owned buffers
  int *h_off = nullptr, *h_idx = nullptr, *c_off = nullptr, *c_idx = nullptr;
  double *Hblk = nullptr, *dHblk = nullptr;
  float* Hsk = nullptr;               // n * max_hnbr * 4: Slater-Koster records (mixed)
  double *lambda = nullptr, *S = nullptr, *P = nullptr;
  int* kdim = nullptr;
  double *mu = nullptr, *ncount = nullptr;
  // launch configuration
  int kry_grid = 0;
  size_t kry_smem = 0;
  int kry_threads = 256;            // threads per Krylov CTA
  bool kry_lsmem = false;           // local CSR of the Krylov kernel in shared memory
  bool ke_on = false;               // persistent Krylov + eigensolve kernel (mixed path)
  int ke_grid = 0;
  size_t ke_smem = 0;
  int ke_ecap = 0;                   // records in shared memory per target (persistent launch)
  int ke_minb = 4;                   // CTAs per SM its register budget allows
  int ke_default_slots = 8;          // records per slot of the default persistent tile
  int sk_ecap = 0;                   // local records kept in shared memory per target
  int sk_grid = 0;                   // CTAs of the mixed Krylov kernel (separate launch)
  size_t sk_smem = 0;
  // launch plan of the mixed Krylov stage: tb_autotune's choice or defaults
  bool tuned = false;
  int plan = 0;                      // tb_schedule in force when schedule == AUTO and tuned
  int plan_nb = 0;                   // buckets of the bucketed plan
  int plan_hi[tb_plan::MAX_BUCKETS] = {};
  tb_sk_cfg plan_cfg[tb_plan::MAX_BUCKETS];
  int* tgt_order = nullptr;          // n: targets by bucket
  int* tgt_boff = nullptr;           // MAX_BINS + 1: bucket offsets
  int* ke_work = nullptr;            // n + 1: work counter, then per-target Krylov-done flags
  int eig_grid = 0;
  int eig_warps = 0;                 // targets per CTA of the warp eigensolver
  size_t eig_smem = 0;
  size_t fin_smem = 0;
  int mu_grid = 0;
  int mu_smem_max = 0;
  // m-target form: grouped block Lanczos, configured when group_m > 1
  int grp_max_union = 0;             // capacity of a group's union cluster
  int grp_grid = 0;
  int grp_mc = 0;                    // targets per CTA (kernel capacity: 2 or 4)
  int grp_threads = 0;
  int grp_ubuf = 0;                  // concatenated member lists (power of two)
  bool grp_vks = false;              // staged copy of V_k in shared memory
  bool grp_lsmem = false;            // local CSR in shared memory
  size_t grp_smem = 0;
  void* grp_V = nullptr;             // grp_grid * grp_mc * r * 16 * max_union (TV)
  int2* grp_lent = nullptr;          // grp_grid * max_union * max_hnbr
  int* grp_cnt = nullptr;            // n: Morton ranks
  int* grp_off = nullptr;            // n + 1: the context's own groups (tb_md_step)
  int* grp_idx = nullptr;            // n
  // exact local gradient: dense workspace, allocated by tb_ctx_reserve_local
  int loc_ND = 0;                    // 4 * max_cluster
  int loc_grid = 0;
  size_t loc_smem = 0;
  size_t loc_esize = 0;              // element size of the dense matrices
  int loc_reserved_n = 0;
  unsigned char* loc_ws = nullptr;
  void *loc_A = nullptr, *loc_Z = nullptr, *loc_X = nullptr;
  double* loc_Cb = nullptr;
  double* loc_Floc = nullptr;
  // stage timing events (tb_profile_enable)
  bool profiling = false;
  bool prof_ran[7] = {false, false, false, false, false, false, false};
  cudaEvent_t prof_ev[14] = {};
};

// Stage timing helpers: record an event pair around a stage when enabled.
tb_status prof_mark(tb_ctx* c, int stage, bool end, cudaStream_t s);

// Launchers (defined in the kernel translation units).
size_t neighbor_cell_capacity(int n);
int neighbor_kernel_count(const tb_ctx* c, double L);
tb_status launch_neighbors(tb_ctx* c, int n, const double* pos, double L, int* h_off,
                           int* h_idx, int* c_off, int* c_idx, cudaStream_t s);
tb_status launch_assemble(tb_ctx* c, int n, const double* pos, double L,
                          const int* h_off, const int* h_idx, double* Hblk,
                          double* dHblk, float* Hsk, cudaStream_t s);
tb_status krylov_configure(tb_ctx* c);
bool krylov_eig_persistent(const tb_ctx* c, int n);   // Krylov launch includes the eigensolve
int krylov_schedule(const tb_ctx* c, int n);          // tb_schedule a launch of n targets uses
int krylov_kernel_count(const tb_ctx* c, int n);      // kernels of the Krylov (+eig) stage
tb_status krylov_autotune(tb_ctx* c, int n, const int* c_off, const int* c_idx, const int* h_off,
                          const int* h_idx, const float* Hsk, double* lambda, double* S,
                          double* P, int* kdim, tb_tune_report* rep, cudaStream_t s);
tb_status launch_krylov(tb_ctx* c, int n, const int* c_off, const int* c_idx,
                        const int* h_off, const int* h_idx, const double* Hblk,
                        const float* Hsk, double* lambda, double* S, double* P, int* kdim,
                        cudaStream_t s);
size_t krylov_overflow_records(const tb_ctx* c);   // records per CTA overflow slot x CTAs
int group_grid_cells(int n, int m);
tb_status krylov_group_configure(tb_ctx* c);
size_t krylov_group_basis_bytes(const tb_ctx* c);
tb_status launch_group_atoms(tb_ctx* c, int n, const double* pos, double L, int* g_off,
                             int* g_idx, cudaStream_t s);
tb_status launch_krylov_grouped(tb_ctx* c, int n, int n_groups, const int* g_off,
                                const int* g_idx, const int* c_off, const int* c_idx,
                                const int* h_off, const int* h_idx, const double* Hblk,
                                const float* Hsk, cudaStream_t s);
tb_status eig_configure(tb_ctx* c);
tb_status launch_eig(tb_ctx* c, int n, const int* h_off, double* lambda, double* S,
                     double* P, int* kdim, cudaStream_t s);
tb_status mu_configure(tb_ctx* c);
tb_status launch_mu(tb_ctx* c, int n, const double* lambda, const double* S,
                    double n_electrons, const double* mu_guess, double* mu,
                    double* n_count, cudaStream_t s);
tb_status launch_forces(tb_ctx* c, int n, const double* pos, double L,
                        const int* h_off, const int* h_idx, const double* dHblk,
                        const double* lambda, const double* S, const double* P,
                        const int* kdim, const double* mu, double* F,
                        double* energies, cudaStream_t s);
tb_status launch_mu_nt(tb_ctx* c, int n, int NT, const double* lambda, const double* S,
                       double n_electrons, const double* mu_guess, double* mu,
                       double* n_count, cudaStream_t s);
tb_status launch_energy_reduce(int n, const double* per_target, const double* mu,
                               double* energies, cudaStream_t s);
tb_status launch_npt_berendsen(tb_ctx* c, int n, double* pos, double* vel, double L,
                               const double* W, const double* energies, double T0, double P0,
                               double dt, double tau_T, double tau_P, double beta,
                               double* L_new, double* state, cudaStream_t s);
tb_status launch_virial(tb_ctx* c, int n, const double* pos, double L, const int* h_off,
                        const int* h_idx, double* W, double* pressure, cudaStream_t s);
tb_status local_configure(tb_ctx* c);
size_t local_workspace_bytes(tb_ctx* c, int n);
void local_carve(tb_ctx* c, int n, unsigned char* base);
tb_status launch_local_forward(tb_ctx* c, int n, const double* pos, double L, const int* c_off,
                               const int* c_idx, const int* h_off, const int* h_idx,
                               const double* Hblk, double* lambda, double* S, int* kdim,
                               void* Zstore, double* mu, double* energies, cudaStream_t s);
tb_status launch_local_gradient(tb_ctx* c, int n, const double* pos, double L, const int* c_off,
                                const int* c_idx, const int* h_off, const int* h_idx,
                                const double* Hblk, const double* dHblk, const double* lambda,
                                const double* S, const void* Zstore, const double* mu, double* F,
                                cudaStream_t s);
tb_status launch_md_kick_drift(tb_ctx* c, int n, double* pos, double* vel,
                               const double* F, double L, double dt, double mass,
                               cudaStream_t s);
tb_status launch_md_kick(tb_ctx* c, int n, double* vel, const double* F,
                         double dt, double mass, double* energies, cudaStream_t s);
