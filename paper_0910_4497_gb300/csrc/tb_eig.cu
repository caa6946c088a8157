// a6-a7: eigenpairs of the projected matrix T (Sec. 3: the small Lanczos
// matrix is diagonalised with a dense symmetric eigensolver) and the spectral
// record lambda, S = U[seed rows], P = Y U.
//
// FP64 arithmetic on this GPU runs at ~1/70 of the FP32 rate with ~70-cycle
// latency, so a serial FP64 tridiagonal QL would dominate the whole force
// evaluation.  The eigensolve is therefore split:
//   1. eig_ql_kernel (one warp per target, FP32): Householder reduction of the
//      active part of T to tridiagonal form with the reflections accumulated,
//      then implicit QL with shifts (Bowdler, Martin, Reinsch & Wilkinson,
//      1968) accumulating the rotations.  Every lane runs the scalar
//      recurrence (identical values), lane 0 stores it, and each lane applies
//      the rotations to its own rows of the eigenvector matrix.
//   2. eig_finish_kernel (one CTA per target):
//      - TB_PREC_MIXED: T itself comes from FP32 sweeps, so the FP32
//        eigenpairs are kept (an FP64 refinement could not add accuracy);
//      - TB_PREC_FP64: two FP64 steps of the Ogita-Aishima refinement
//        (Japan J. Indust. Appl. Math. 35 (2018)): R = I - X^T X,
//        S = X^T T X, lambda_i = S_ii/(1 - R_ii), E_ij = (S_ij + lambda_j R_ij)
//        /(lambda_j - lambda_i) if the gap exceeds delta else R_ij/2,
//        X <- X + X E, then FP64 Rayleigh quotients;
//      then the eigenpairs are sorted ascending and S, P are formed.
#include "tb_internal.cuh"

namespace {

constexpr int EW = 4;              // warps (targets) per CTA in the QL kernel
constexpr int FT = 128;            // threads per CTA in the finishing kernel

struct EigArgs {
  int n, NT;
  const double* T;
  const unsigned long long* colmask;
  float* Zf;
  float* lamf;
  int* kdim;
  int* st;
};

__host__ __device__ inline int pitch_of(int NT) { return NT + 1; }

__host__ __device__ inline size_t ql_smem_per_warp(int NT) {
  // Z (NT x (NT+1) floats: the matrix, then the Householder vectors, then the
  // eigenvectors), v, q, d, e (NT floats), act (NT ints)
  return sizeof(float) * ((size_t)NT * pitch_of(NT) + 4 * NT) + sizeof(int) * NT;
}

__global__ void __launch_bounds__(EW * 32) eig_ql_kernel(const EigArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int NT = a.NT, PT = pitch_of(NT);
  unsigned char* base = smem + warp * ql_smem_per_warp(NT);
  float* Z = reinterpret_cast<float*>(base);
  float* vv = Z + NT * PT;
  float* qq = vv + NT;
  float* d = qq + NT;
  float* e = d + NT;
  int* act = reinterpret_cast<int*>(e + NT);
  const int i = blockIdx.x * EW + warp;
  if (i >= a.n) return;

  const unsigned long long mask = a.colmask[i];
  const int m = __popcll(mask);
  for (int x = lane; x < NT; x += 32)
    if ((mask >> x) & 1ull) act[__popcll(mask & ((1ull << x) - 1ull))] = x;
  __syncwarp();
  const double* Ti = a.T + (size_t)i * NT * NT;
  for (int x = 0; x < m; ++x)
    for (int y = lane; y < m; y += 32) Z[x * PT + y] = (float)Ti[act[x] * NT + act[y]];
  __syncwarp();

  // ---- Householder reduction to tridiagonal form.  Step j zeroes column j
  // below the subdiagonal with H_j = I - 2 v v^T (v supported on rows > j) and
  // stores v in that column; each lane owns rows x = lane, lane + 32.
  for (int j = 0; j + 2 < m; ++j) {
    float xs = 0.f;
    for (int x = lane; x < m; x += 32)
      if (x > j) xs += Z[x * PT + j] * Z[x * PT + j];
    const float sig = tbk::warp_sum(xs);
    const float x0 = Z[(j + 1) * PT + j];
    __syncwarp();
    if (sig - x0 * x0 <= 1e-30f * (sig + 1e-30f) || sig == 0.f) {
      if (lane == 0) e[j] = x0;
      for (int x = lane; x < m; x += 32)
        if (x > j) Z[x * PT + j] = 0.f;      // identity reflection
      __syncwarp();
      continue;
    }
    const float alpha = x0 >= 0.f ? -sqrtf(sig) : sqrtf(sig);
    const float inv = rsqrtf(2.f * (sig - x0 * alpha));
    for (int x = lane; x < m; x += 32)
      vv[x] = x <= j ? 0.f : (x == j + 1 ? (x0 - alpha) : Z[x * PT + j]) * inv;
    __syncwarp();
    float kp = 0.f;
    for (int x = lane; x < m; x += 32) {
      float p = 0.f;
      if (x > j)
        for (int l = j + 1; l < m; ++l) p += Z[x * PT + l] * vv[l];
      qq[x] = p;
      kp += p * vv[x];
    }
    const float K = tbk::warp_sum(kp);
    for (int x = lane; x < m; x += 32) qq[x] -= K * vv[x];
    __syncwarp();
    for (int x = lane; x < m; x += 32) {
      if (x > j) {
        const float vx = vv[x], qx = qq[x];
        for (int l = j + 1; l < m; ++l) Z[x * PT + l] -= 2.f * (vx * qq[l] + qx * vv[l]);
        Z[x * PT + j] = vx;                  // keep v_j in column j
      }
    }
    if (lane == 0) e[j] = alpha;
    __syncwarp();
  }
  for (int x = lane; x < m; x += 32) d[x] = Z[x * PT + x];
  if (lane == 0) {
    if (m >= 2) e[m - 2] = Z[(m - 1) * PT + (m - 2)];
    if (m >= 1) e[m - 1] = 0.f;
  }
  __syncwarp();
  // ---- accumulate Q = H_0 H_1 ... H_{m-3} in place, last reflection first;
  // lanes own columns l = lane, lane + 32.
  // Invariant: before applying H_j, the block of rows and columns > j holds
  // H_{j+1} ... H_{m-3} restricted to those indices; entries left of that block
  // still hold the reflection vectors.  Start from the trailing identity.
  if (lane == 0) {
    const int t0 = m >= 2 ? m - 2 : 0;
    for (int x = t0; x < m; ++x)
      for (int y = t0; y < m; ++y) Z[x * PT + y] = (x == y) ? 1.f : 0.f;
  }
  __syncwarp();
  for (int j = m - 3; j >= 0; --j) {
    for (int x = lane; x < m; x += 32) vv[x] = x > j ? Z[x * PT + j] : 0.f;
    __syncwarp();
    for (int l = lane; l < m; l += 32) {
      if (l > j) {
        float sl = 0.f;
        for (int y = j + 1; y < m; ++y) sl += vv[y] * Z[y * PT + l];
        sl *= 2.f;
        for (int y = j + 1; y < m; ++y) Z[y * PT + l] -= sl * vv[y];
      }
    }
    __syncwarp();
    for (int x = lane; x < m; x += 32) {
      if (x >= j) {
        Z[x * PT + j] = (x == j) ? 1.f : 0.f;
        Z[j * PT + x] = (x == j) ? 1.f : 0.f;
      }
    }
    __syncwarp();
  }

  // ---- implicit QL with shifts on (d, e); rotations applied to the rows of Z.
  // Rotation (c, s) from f, g via one reciprocal square root.
  float tn = 0.f;
  for (int x = lane; x < m; x += 32) tn = fmaxf(tn, fabsf(d[x]) + fabsf(e[x]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tn = fmaxf(tn, __shfl_xor_sync(0xffffffffu, tn, o));
  // deflate an off-diagonal once it is a few FP32 ulps of ||T||: below that the
  // rotations only churn rounding noise
  const float tol = 4.8e-7f * tn;
  bool failed = false;
  for (int l = 0; l < m; ++l) {
    int iter = 0;
    while (true) {
      int mm = l;
      while (mm < m - 1 && fabsf(e[mm]) > tol) ++mm;
      if (mm == l) break;
      if (++iter > 60) { failed = true; break; }
      const float el = e[l], dl = d[l];
      float g = (d[l + 1] - dl) / (2.f * el);
      float rr = sqrtf(g * g + 1.f);
      g = d[mm] - dl + el / (g + (g >= 0.f ? rr : -rr));
      float s = 1.f, c = 1.f, p = 0.f;
      bool early = false;
      for (int ii = mm - 1; ii >= l; --ii) {
        const float ei = e[ii], di = d[ii], di1 = d[ii + 1];
        const float f = s * ei, b = c * ei;
        const float h = f * f + g * g;
        __syncwarp();
        if (h == 0.f) {
          if (lane == 0) { e[ii + 1] = 0.f; d[ii + 1] = di1 - p; e[mm] = 0.f; }
          early = true;
          break;
        }
        const float rinv = rsqrtf(h);
        if (lane == 0) e[ii + 1] = h * rinv;
        s = f * rinv;
        c = g * rinv;
        g = di1 - p;
        rr = (di - g) * s + 2.f * c * b;
        p = s * rr;
        if (lane == 0) d[ii + 1] = g + p;
        g = c * rr - b;
        for (int x = lane; x < m; x += 32) {
          const float z1 = Z[x * PT + ii + 1], z0 = Z[x * PT + ii];
          Z[x * PT + ii + 1] = s * z0 + c * z1;
          Z[x * PT + ii] = c * z0 - s * z1;
        }
      }
      __syncwarp();
      if (!early) {
        if (lane == 0) { d[l] = d[l] - p; e[l] = g; e[mm] = 0.f; }
      }
      __syncwarp();
    }
    if (failed) break;
  }
  if (failed && lane == 0) tbk::set_status(a.st, TB_ERR_NO_CONVERGENCE, i);
  float* lf = a.lamf + (size_t)i * NT;
  float* zo = a.Zf + (size_t)i * NT * NT;
  for (int x = lane; x < m; x += 32) lf[x] = d[x];
  for (int x = 0; x < m; ++x)
    for (int y = lane; y < m; y += 32) zo[x * NT + y] = Z[x * PT + y];
  if (lane == 0) a.kdim[i] = m;
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
  if (sizeof(TV) == sizeof(float)) {
    b += sizeof(float) * NT * PT;           // X
  } else {
    b += sizeof(double) * NT * PT * 5;      // T, X, W1, Smat, Rmat
  }
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

  if (sizeof(TV) == sizeof(float)) {
    // T comes from FP32 sweeps and is FP32-accurate: the FP32 QL eigenvalues
    // already carry the full accuracy available.
    for (int k = tid; k < m; k += FT) lam[k] = (double)a.lamf[(size_t)i * NT + k];
    __syncthreads();
  } else {
    const double* Ti = a.T + (size_t)i * NT * NT;
    double* Xd = reinterpret_cast<double*>(X);
    double* Tm = Xd + NT * PT;
    double* W1 = Tm + NT * PT;
    double* Sm = W1 + NT * PT;
    double* Rm = Sm + NT * PT;
    for (int q = tid; q < m * m; q += FT) {
      const int x = q / m, y = q - x * m;
      Tm[x * PT + y] = Ti[act[x] * NT + act[y]];
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

}  // namespace

tb_status eig_configure(tb_ctx* c) {
  const int NT = 4 * c->p.r;
  c->eig_smem = EW * ql_smem_per_warp(NT);
  TB_CUDA_TRY(cudaFuncSetAttribute(eig_ql_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   (int)c->eig_smem));
  if (c->p.prec == TB_PREC_FP64) {
    c->fin_smem = fin_smem_bytes<double>(NT);
    TB_CUDA_TRY(cudaFuncSetAttribute(eig_finish_kernel<double>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->fin_smem));
  } else {
    c->fin_smem = fin_smem_bytes<float>(NT);
    TB_CUDA_TRY(cudaFuncSetAttribute(eig_finish_kernel<float>,
                                     cudaFuncAttributeMaxDynamicSharedMemorySize, (int)c->fin_smem));
  }
  return TB_OK;
}

tb_status launch_eig(tb_ctx* c, int n, const int* h_off, double* lambda, double* S,
                     double* P, int* kdim, cudaStream_t s) {
  if (n <= 0) return TB_OK;
  const int NT = 4 * c->p.r;
  EigArgs ea{n, NT, c->T, c->colmask, c->Zf, c->lamf, kdim, c->d_status};
  eig_ql_kernel<<<(n + EW - 1) / EW, EW * 32, c->eig_smem, s>>>(ea);
  TB_CUDA_TRY(cudaGetLastError());
  if (c->p.prec == TB_PREC_FP64) {
    FinArgs<double> fa{n, NT, c->T, c->colmask, c->Zf, c->lamf,
                       reinterpret_cast<const double*>(c->Y), h_off, lambda, S, P, c->d_status};
    eig_finish_kernel<double><<<n, FT, c->fin_smem, s>>>(fa);
  } else {
    FinArgs<float> fa{n, NT, c->T, c->colmask, c->Zf, c->lamf,
                      reinterpret_cast<const float*>(c->Y), h_off, lambda, S, P, c->d_status};
    eig_finish_kernel<float><<<n, FT, c->fin_smem, s>>>(fa);
  }
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}
