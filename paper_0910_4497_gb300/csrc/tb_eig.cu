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
//      - TB_PREC_MIXED: FP64 Rayleigh quotients lambda_k = x_k^T T x_k /
//        x_k^T x_k on the FP32 eigenvectors (eigenvalue error second order in
//        the eigenvector error);
//      - TB_PREC_FP64: two FP64 iterations of the Ogita-Aishima refinement
//        (Japan J. Indust. Appl. Math. 35 (2018)): R = I - X^T X,
//        S = X^T T X, lambda_i = S_ii/(1 - R_ii), E_ij = (S_ij + lambda_j R_ij)
//        /(lambda_j - lambda_i) if the gap exceeds delta else R_ij/2,
//        X <- X + X E.
//      then the eigenpairs are sorted ascending and S, P are formed.
#include "tb_internal.cuh"

namespace {

constexpr int EW = 2;              // warps (targets) per CTA in the QL kernel
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
  // A and Z (NT x (NT+1) floats), v, q, d, e (NT floats), act (NT ints)
  return sizeof(float) * (2 * (size_t)NT * pitch_of(NT) + 4 * NT) + sizeof(int) * NT;
}

__global__ void __launch_bounds__(EW * 32) eig_ql_kernel(const EigArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int NT = a.NT, PT = pitch_of(NT);
  unsigned char* base = smem + warp * ql_smem_per_warp(NT);
  float* A = reinterpret_cast<float*>(base);
  float* Z = A + NT * PT;
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
    for (int y = lane; y < m; y += 32) {
      A[x * PT + y] = (float)Ti[act[x] * NT + act[y]];
      Z[x * PT + y] = (x == y) ? 1.f : 0.f;
    }
  __syncwarp();

  // ---- Householder tridiagonalisation, reflections accumulated into Z
  for (int j = 0; j + 2 < m; ++j) {
    float xs = 0.f;
    for (int x = lane; x < m; x += 32)
      if (x > j) xs += A[x * PT + j] * A[x * PT + j];
    const float sig = tbk::warp_sum(xs);
    const float x0 = A[(j + 1) * PT + j];
    if (sig - x0 * x0 <= 1e-30f * (sig + 1e-30f) || sig == 0.f) {
      if (lane == 0) e[j] = x0;
      __syncwarp();
      continue;
    }
    const float alpha = x0 >= 0.f ? -sqrtf(sig) : sqrtf(sig);
    const float inv = rsqrtf(2.f * (sig - x0 * alpha));
    for (int x = lane; x < m; x += 32)
      vv[x] = x <= j ? 0.f : (x == j + 1 ? (x0 - alpha) : A[x * PT + j]) * inv;
    __syncwarp();
    float kp = 0.f;
    for (int x = lane; x < m; x += 32) {
      float p = 0.f;
      if (x > j)
        for (int l = j + 1; l < m; ++l) p += A[x * PT + l] * vv[l];
      qq[x] = p;
      kp += p * vv[x];
    }
    const float K = tbk::warp_sum(kp);
    for (int x = lane; x < m; x += 32) qq[x] -= K * vv[x];
    __syncwarp();
    for (int x = lane; x < m; x += 32) {
      if (x > j) {
        const float vx = vv[x], qx = qq[x];
        for (int l = j + 1; l < m; ++l) A[x * PT + l] -= 2.f * (vx * qq[l] + qx * vv[l]);
      }
      float t = 0.f;
      for (int l = j + 1; l < m; ++l) t += Z[x * PT + l] * vv[l];
      for (int l = j + 1; l < m; ++l) Z[x * PT + l] -= 2.f * t * vv[l];
    }
    if (lane == 0) e[j] = alpha;
    __syncwarp();
  }
  for (int x = lane; x < m; x += 32) d[x] = A[x * PT + x];
  if (lane == 0) {
    if (m >= 2) e[m - 2] = A[(m - 1) * PT + (m - 2)];
    if (m >= 1) e[m - 1] = 0.f;
  }
  __syncwarp();

  // ---- implicit QL with shifts on (d, e), rotations applied to the rows of Z
  float tn = 0.f;
  for (int x = lane; x < m; x += 32) tn = fmaxf(tn, fabsf(d[x]) + fabsf(e[x]));
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) tn = fmaxf(tn, __shfl_xor_sync(0xffffffffu, tn, o));
  const float tol = 1.2e-7f * tn;
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
        rr = sqrtf(f * f + g * g);
        __syncwarp();
        if (lane == 0) e[ii + 1] = rr;
        if (rr == 0.f) {
          if (lane == 0) { d[ii + 1] = di1 - p; e[mm] = 0.f; }
          early = true;
          break;
        }
        s = f / rr;
        c = g / rr;
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
  size_t b = sizeof(int) * 2 * NT + sizeof(double) * 4 * NT;   // act, blk; lam, rank, misc
  if (sizeof(TV) == sizeof(float)) {
    b += sizeof(double) * NT * PT;          // T active
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
  double* lam = reinterpret_cast<double*>(rank + NT);
  double* red = lam + NT;          // 3*NT doubles of scratch
  double* Tm = red + 3 * NT;
  const unsigned long long mask = a.colmask[i];
  const int m = __popcll(mask);
  for (int x = tid; x < NT; x += FT)
    if ((mask >> x) & 1ull) act[__popcll(mask & ((1ull << x) - 1ull))] = x;
  __syncthreads();
  const double* Ti = a.T + (size_t)i * NT * NT;
  for (int q = tid; q < m * m; q += FT) {
    const int x = q / m, y = q - x * m;
    Tm[x * PT + y] = Ti[act[x] * NT + act[y]];
  }
  const float* Zi = a.Zf + (size_t)i * NT * NT;
  TV* X = reinterpret_cast<TV*>(Tm + NT * PT);
  for (int q = tid; q < m * m; q += FT) {
    const int x = q / m, y = q - x * m;
    X[x * PT + y] = (TV)Zi[x * NT + y];
  }
  __syncthreads();
  // active columns x, y couple only if their Krylov blocks are adjacent
  auto near = [&](int x, int y) { int bx = act[x] >> 2, by = act[y] >> 2; return bx - by <= 1 && by - bx <= 1; };

  if (sizeof(TV) == sizeof(float)) {
    for (int k = tid; k < m; k += FT) {
      double num = 0.0, den = 0.0;
      for (int x = 0; x < m; ++x) {
        const double xk = (double)X[x * PT + k];
        double t = 0.0;
        for (int y = 0; y < m; ++y)
          if (near(x, y)) t += Tm[x * PT + y] * (double)X[y * PT + k];
        num += xk * t;
        den += xk * xk;
      }
      lam[k] = num / den;
    }
    __syncthreads();
  } else {
    double* Xd = reinterpret_cast<double*>(X);
    double* W1 = Xd + NT * PT;
    double* Sm = W1 + NT * PT;
    double* Rm = Sm + NT * PT;
    // ||T||_F
    if (tid == 0) {
      double t2 = 0.0;
      for (int q = 0; q < m * m; ++q) { const double v = Tm[(q / m) * PT + q % m]; t2 += v * v; }
      red[0] = sqrt(t2);
    }
    __syncthreads();
    const double tnorm = red[0];
    for (int it = 0; it < 2; ++it) {
      for (int q = tid; q < m * m; q += FT) {           // W1 = T X (banded T)
        const int x = q / m, k = q - x * m;
        double t = 0.0;
        for (int y = 0; y < m; ++y) if (near(x, y)) t += Tm[x * PT + y] * Xd[y * PT + k];
        W1[x * PT + k] = t;
      }
      __syncthreads();
      for (int q = tid; q < m * m; q += FT) {           // S = X^T W1, R = I - X^T X
        const int x = q / m, y = q - x * m;
        double s = 0.0, rr = 0.0;
        for (int l = 0; l < m; ++l) {
          s += Xd[l * PT + x] * W1[l * PT + y];
          rr += Xd[l * PT + x] * Xd[l * PT + y];
        }
        Sm[x * PT + y] = s;
        Rm[x * PT + y] = (x == y ? 1.0 : 0.0) - rr;
      }
      __syncthreads();
      for (int k = tid; k < m; k += FT) lam[k] = Sm[k * PT + k] / (1.0 - Rm[k * PT + k]);
      __syncthreads();
      if (tid == 0) {
        double so = 0.0, ro = 0.0;
        for (int q = 0; q < m * m; ++q) {
          const int x = q / m, y = q - x * m;
          const double sv = Sm[x * PT + y] - (x == y ? lam[x] : 0.0);
          so += sv * sv;
          ro += Rm[x * PT + y] * Rm[x * PT + y];
        }
        red[1] = 2.0 * (sqrt(so) + tnorm * sqrt(ro));
      }
      __syncthreads();
      const double delta = red[1];
      for (int q = tid; q < m * m; q += FT) {           // E overwrites S
        const int x = q / m, y = q - x * m;
        double ev;
        if (x == y) ev = 0.5 * Rm[x * PT + y];
        else {
          const double gap = lam[y] - lam[x];
          ev = fabs(gap) > delta ? (Sm[x * PT + y] + lam[y] * Rm[x * PT + y]) / gap
                                 : 0.5 * Rm[x * PT + y];
        }
        W1[x * PT + y] = ev;
      }
      __syncthreads();
      for (int q = tid; q < m * m; q += FT) {           // X + X E  -> S
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
    // final Rayleigh quotients on the refined vectors
    for (int k = tid; k < m; k += FT) {
      double num = 0.0, den = 0.0;
      for (int x = 0; x < m; ++x) {
        double t = 0.0;
        for (int y = 0; y < m; ++y) if (near(x, y)) t += Tm[x * PT + y] * Xd[y * PT + k];
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
    double out = 0.0;
    if (k < m) {
      const TV* yr = a.Y + (rbase + rr) * NT;
      TV t = (TV)0;
      for (int l = 0; l < m; ++l) t += yr[act[l]] * X[l * PT + k];
      out = (double)t;
      a.P[(rbase + rr) * NT + rank[k]] = out;
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
