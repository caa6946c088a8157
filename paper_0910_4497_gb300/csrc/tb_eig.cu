// Eigenpairs of the projected matrix T (Sec. 3: the small Lanczos
// matrix is diagonalised with a dense symmetric eigensolver) and the spectral
// record lambda, S = U[seed rows], P = Y U.
//
// FP64 arithmetic on this GPU runs at ~1/70 of the FP32 rate with ~70-cycle
// latency, so the eigensolve runs in FP32 with FP64-accurate corrections:
//   eig_warp_kernel: one 64-thread group per target, up to five per CTA, each
//   running the group eigensolver of tb_eig_group.cuh (Householder,
//   bisection, twisted-factorisation eigenvectors, back-transformation; in
//   the mixed path also the Loewdin step, double-float Rayleigh quotients and
//   the spectral record);
//   in the FP64 path the FP32 eigenpairs go to eig_finish_kernel<double>:
//      two FP64 steps of the Ogita-Aishima refinement
//      (Japan J. Indust. Appl. Math. 35 (2018)): R = I - X^T X,
//      S = X^T T X, lambda_i = S_ii/(1 - R_ii), E_ij = (S_ij + lambda_j R_ij)
//      /(lambda_j - lambda_i) if the gap exceeds delta else R_ij/2,
//      X <- X + X E, then FP64 Rayleigh quotients, ascending order, S and P.
#include "tb_internal.cuh"
#include "tb_eig_group.cuh"

namespace {

constexpr int FT = 128;            // threads per CTA in the finishing kernel
constexpr int XW_MAX = 5;          // targets (64-thread groups) per CTA in eig_warp_kernel

// (64-wide rows: three targets per CTA by shared memory, so a looser register cap)
template <bool FULL, int NTC>
__global__ void __launch_bounds__(XW_MAX * GT, NTC == 64 ? 1 : 2) eig_warp_kernel(const XArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int grp = threadIdx.x / GT;
  Grp g;
  g.t = threadIdx.x % GT;
  g.wl = threadIdx.x & 31;
  g.gw = g.t >> 5;
  g.bid = 1 + grp;
  const int i = blockIdx.x * (blockDim.x / GT) + grp;
  if (i >= a.n) return;                       // whole group: no block barriers below
  eig_group<FULL, NTC>(a, i, g, smem + grp * xw_smem_per_warp(a.NT));
}

// ------------------------------------------------------------------ finishing

template <typename TV>
struct FinArgs {
  int n, NT;
  const double* T;
  const unsigned long long* colmask;
  const float* Zf;
  const float* lamf;
  const TV* Y;
  const int* h_off;
  double* lambda;
  double* S;
  double* P;
  int* st;
};

template <typename TV>
__host__ __device__ inline size_t fin_smem_bytes(int NT) {
  const size_t PT = NT + 1;
  size_t b = sizeof(int) * 4 * NT + sizeof(double) * 4 * NT;   // act, rank, lo, hi; lam, red
  b += sizeof(double) * NT * PT * 5;                           // T, X, W1, Smat, Rmat
  return b + 64;
}

template <typename TV>
__global__ void __launch_bounds__(FT) eig_finish_kernel(const FinArgs<TV> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x;
  const int NT = a.NT, PT = NT + 1;
  const int i = blockIdx.x;
  int* act = reinterpret_cast<int*>(smem);
  int* rank = act + NT;
  int* blo = rank + NT;             // band of row x in compacted indices: [blo, bhi)
  int* bhi = blo + NT;
  double* lam = reinterpret_cast<double*>(bhi + NT);
  double* red = lam + NT;           // 3*NT doubles of scratch
  TV* X = reinterpret_cast<TV*>(red + 3 * NT);
  const unsigned long long mask = a.colmask[i];
  const int m = __popcll(mask);
  for (int x = tid; x < NT; x += FT)
    if ((mask >> x) & 1ull) act[__popcll(mask & ((1ull << x) - 1ull))] = x;
  __syncthreads();
  // active columns couple in T only when their Krylov blocks are adjacent
  for (int x = tid; x < m; x += FT) {
    const int bx = act[x] >> 2;
    int lo = x, hi = x + 1;
    while (lo > 0 && (act[lo - 1] >> 2) >= bx - 1) --lo;
    while (hi < m && (act[hi] >> 2) <= bx + 1) ++hi;
    blo[x] = lo;
    bhi[x] = hi;
  }
  const float* Zi = a.Zf + (size_t)i * NT * NT;
  for (int q = tid; q < m * m; q += FT) {
    const int x = q / m, y = q - x * m;
    X[x * PT + y] = (TV)Zi[x * NT + y];
  }
  __syncthreads();

  {
  const double* Ti = a.T + (size_t)i * tc_doubles(NT / 4);
  double* Xd = reinterpret_cast<double*>(X);
  double* Tm = Xd + NT * PT;
  double* W1 = Tm + NT * PT;
  double* Sm = W1 + NT * PT;
  double* Rm = Sm + NT * PT;
  for (int q = tid; q < m * m; q += FT) {
    const int x = q / m, y = q - x * m;
    const int tq = tc_index(act[x], act[y]);
    Tm[x * PT + y] = tq < 0 ? 0.0 : Ti[tq];
  }
  __syncthreads();
  {
    double t2 = 0.0;
    for (int q = tid; q < m * m; q += FT) {
      const double v = Tm[(q / m) * PT + q % m];
      t2 += v * v;
    }
    double v1[1] = {t2};
    tbk::block_sum<double, 1>(v1, red, red + 2 * NT);
  }
  const double tnorm = sqrt(red[2 * NT]);
  // two Ogita-Aishima refinement steps (quadratic convergence from FP32; the
  // second resolves near-degenerate pairs the first one leaves mixed)
  for (int it = 0; it < 2; ++it) {
  for (int q = tid; q < m * m; q += FT) {           // W1 = T X (banded T)
    const int x = q / m, k = q - x * m;
    double t = 0.0;
    for (int y = blo[x]; y < bhi[x]; ++y) t += Tm[x * PT + y] * Xd[y * PT + k];
    W1[x * PT + k] = t;
  }
  __syncthreads();
  for (int q = tid; q < m * m; q += FT) {           // S = X^T W1, R = I - X^T X
    const int x = q / m, y = q - x * m;
    double sv = 0.0, rr = 0.0;
    for (int l = 0; l < m; ++l) {
      sv += Xd[l * PT + x] * W1[l * PT + y];
      rr += Xd[l * PT + x] * Xd[l * PT + y];
    }
    Sm[x * PT + y] = sv;
    Rm[x * PT + y] = (x == y ? 1.0 : 0.0) - rr;
  }
  __syncthreads();
  for (int k = tid; k < m; k += FT) lam[k] = Sm[k * PT + k] / (1.0 - Rm[k * PT + k]);
  __syncthreads();
  {
    double so = 0.0, ro = 0.0;
    for (int q = tid; q < m * m; q += FT) {
      const int x = q / m, y = q - x * m;
      const double sv = Sm[x * PT + y] - (x == y ? lam[x] : 0.0);
      so += sv * sv;
      ro += Rm[x * PT + y] * Rm[x * PT + y];
    }
    double v2[2] = {so, ro};
    tbk::block_sum<double, 2>(v2, red, red + 2 * NT);
  }
  const double delta = 2.0 * (sqrt(red[2 * NT]) + tnorm * sqrt(red[2 * NT + 1]));
  for (int q = tid; q < m * m; q += FT) {           // E
    const int x = q / m, y = q - x * m;
    double ev;
    if (x == y) {
      ev = 0.5 * Rm[x * PT + y];
    } else {
      const double gap = lam[y] - lam[x];
      ev = fabs(gap) > delta ? (Sm[x * PT + y] + lam[y] * Rm[x * PT + y]) / gap
                             : 0.5 * Rm[x * PT + y];
    }
    W1[x * PT + y] = ev;
  }
  __syncthreads();
  for (int q = tid; q < m * m; q += FT) {           // X + X E -> S
    const int x = q / m, y = q - x * m;
    double t = Xd[x * PT + y];
    for (int l = 0; l < m; ++l) t += Xd[x * PT + l] * W1[l * PT + y];
    Sm[x * PT + y] = t;
  }
  __syncthreads();
  for (int q = tid; q < m * m; q += FT) {
    const int x = q / m, y = q - x * m;
    Xd[x * PT + y] = Sm[x * PT + y];
  }
  __syncthreads();
  }
  // Rayleigh quotients on the refined vectors
  for (int k = tid; k < m; k += FT) {
    double num = 0.0, den = 0.0;
    for (int x = 0; x < m; ++x) {
      double t = 0.0;
      for (int y = blo[x]; y < bhi[x]; ++y) t += Tm[x * PT + y] * Xd[y * PT + k];
      num += Xd[x * PT + k] * t;
      den += Xd[x * PT + k] * Xd[x * PT + k];
    }
    lam[k] = num / den;
  }
  __syncthreads();
  }
  // ---- ascending order (ties by index)
  for (int k = tid; k < m; k += FT) {
    int rk = 0;
    const double lk = lam[k];
    for (int q = 0; q < m; ++q) rk += (lam[q] < lk) || (lam[q] == lk && q < k);
    rank[k] = rk;
    if (!isfinite(lk)) tbk::set_status(a.st, TB_ERR_NONFINITE, i);
  }
  __syncthreads();
  double* lo = a.lambda + (size_t)i * NT;
  for (int k = tid; k < NT; k += FT) if (k >= m) lo[k] = 0.0;
  for (int k = tid; k < m; k += FT) lo[rank[k]] = lam[k];
  double* So = a.S + (size_t)i * 4 * NT;
  for (int q = tid; q < 4 * NT; q += FT) {
    const int al = q / NT, k = q - al * NT;
    if (k >= m) So[al * NT + k] = 0.0;
  }
  for (int q = tid; q < 4 * m; q += FT) {
    const int al = q / m, k = q - al * m;
    So[al * NT + rank[k]] = (double)X[al * PT + k];
  }
  // P = Y[:, active] X
  const int deg = a.h_off[i + 1] - a.h_off[i];
  const size_t rbase = (size_t)(i + a.h_off[i]) * 4;
  const int nrows = 4 * (deg + 1);
  for (int q = tid; q < nrows * NT; q += FT) {
    const int rr = q / NT, k = q - rr * NT;
    if (k < m) {
      const TV* yr = a.Y + (rbase + rr) * NT;
      TV t = (TV)0;
      for (int l = 0; l < m; ++l) t += yr[act[l]] * X[l * PT + k];
      a.P[(rbase + rr) * NT + rank[k]] = (double)t;
    } else {
      a.P[(rbase + rr) * NT + k] = 0.0;
    }
  }
}

template <bool FULL>
cudaError_t eig_set_smem(int NT, int bytes) {
  const int ntc = ntc_of(NT);
  auto attr = cudaFuncAttributeMaxDynamicSharedMemorySize;
  if (ntc == 16) return cudaFuncSetAttribute(eig_warp_kernel<FULL, 16>, attr, bytes);
  if (ntc == 32) return cudaFuncSetAttribute(eig_warp_kernel<FULL, 32>, attr, bytes);
  if (ntc == 48) return cudaFuncSetAttribute(eig_warp_kernel<FULL, 48>, attr, bytes);
  return cudaFuncSetAttribute(eig_warp_kernel<FULL, 64>, attr, bytes);
}

template <bool FULL>
void eig_launch(int NT, int grid, int threads, size_t smem, cudaStream_t s, const XArgs& xa) {
  const int ntc = ntc_of(NT);
  if (ntc == 16) eig_warp_kernel<FULL, 16><<<grid, threads, smem, s>>>(xa);
  else if (ntc == 32) eig_warp_kernel<FULL, 32><<<grid, threads, smem, s>>>(xa);
  else if (ntc == 48) eig_warp_kernel<FULL, 48><<<grid, threads, smem, s>>>(xa);
  else eig_warp_kernel<FULL, 64><<<grid, threads, smem, s>>>(xa);
}

}  // namespace

tb_status eig_configure(tb_ctx* c) {
  const int NT = 4 * c->p.r;
  const size_t per = xw_smem_per_warp(NT);
  int sm_smem = 0;
  TB_CUDA_TRY(cudaDeviceGetAttribute(&sm_smem, cudaDevAttrMaxSharedMemoryPerMultiprocessor,
                                     c->device));
  int xw = (int)((size_t)(sm_smem / 2 - 1024) / per);   // targets per CTA; two CTAs per SM
  if (xw > XW_MAX) xw = XW_MAX;
  if (xw < 1) xw = 1;
  if (NT > GT) return TB_ERR_CAPACITY;
  c->eig_warps = xw;
  c->eig_smem = xw * per;
  if (c->p.prec == TB_PREC_FP64) {
    TB_CUDA_TRY(eig_set_smem<false>(NT, (int)c->eig_smem));
    c->fin_smem = fin_smem_bytes<double>(NT);
    TB_CUDA_TRY(cudaFuncSetAttribute(eig_finish_kernel<double>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->fin_smem));
  } else {
    TB_CUDA_TRY(eig_set_smem<true>(NT, (int)c->eig_smem));
  }
  return TB_OK;
}

tb_status launch_eig(tb_ctx* c, int n, const int* h_off, double* lambda, double* S,
                     double* P, int* kdim, cudaStream_t s) {
  if (n <= 0) return TB_OK;
  const int NT = 4 * c->p.r;
  if (krylov_eig_persistent(c, n)) return TB_OK;      // done in the Krylov launch
  const int xw = c->eig_warps;
  XArgs xa{n, NT, c->T, c->colmask, reinterpret_cast<const float*>(c->Y), h_off, c->Zf,
           c->lamf, lambda, S, P, kdim, c->d_status};
  if (c->p.prec == TB_PREC_FP64) {
    eig_launch<false>(NT, (n + xw - 1) / xw, xw * GT, c->eig_smem, s, xa);
    TB_CUDA_TRY(cudaGetLastError());
    FinArgs<double> fa{n, NT, c->T, c->colmask, c->Zf, c->lamf,
                       reinterpret_cast<const double*>(c->Y), h_off, lambda, S, P, c->d_status};
    eig_finish_kernel<double><<<n, FT, c->fin_smem, s>>>(fa);
  } else {
    eig_launch<true>(NT, (n + xw - 1) / xw, xw * GT, c->eig_smem, s, xa);
  }
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}
