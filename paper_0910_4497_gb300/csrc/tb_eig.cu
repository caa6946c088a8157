// a6-a7: eigenpairs of the projected matrix T (Sec. 3: the small Lanczos
// matrix is diagonalised with a dense symmetric eigensolver) and the spectral
// record lambda, S = U[seed rows], P = Y U.
//
// FP64 arithmetic on this GPU runs at ~1/70 of the FP32 rate with ~70-cycle
// latency, so a serial FP64 tridiagonal QL would dominate the whole force
// evaluation.  The eigensolve is therefore split:
//   1. eig_tri_kernel (one warp per target, FP32): Householder reduction of
//      the active part of T to tridiagonal form; eigenvalues by Sturm-sequence
//      bisection, each lane owning its own eigenvalues; eigenvectors by
//      inverse iteration (tridiagonal LU with partial pivoting, three solves),
//      lane-parallel, with Gram-Schmidt inside clusters of eigenvalues closer
//      than 1e-3 ||T|| after every solve (the scheme of LAPACK's stein);
//      back-transformation through the stored reflections.
//   2. eig_finish_kernel (one CTA per target):
//      - TB_PREC_MIXED: a first-order Loewdin step makes the FP32 eigenvectors
//        orthonormal, then FP64 Rayleigh quotients give the eigenvalues;
//      - TB_PREC_FP64: two FP64 steps of the Ogita-Aishima refinement
//        (Japan J. Indust. Appl. Math. 35 (2018)): R = I - X^T X,
//        S = X^T T X, lambda_i = S_ii/(1 - R_ii), E_ij = (S_ij + lambda_j R_ij)
//        /(lambda_j - lambda_i) if the gap exceeds delta else R_ij/2,
//        X <- X + X E, then FP64 Rayleigh quotients;
//      then the eigenpairs are sorted ascending and S, P are formed.
#include "tb_internal.cuh"

namespace {

constexpr int EW = 4;              // warps (targets) per CTA in the eigensolver
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

// Row pitch of the per-warp matrices: a multiple of 4 (float4 rows) whose
// stride in banks keeps 8 consecutive rows' 16-byte accesses conflict-free.
__host__ __device__ inline int pitch_of(int NT) { return NT + 4; }

__host__ __device__ inline size_t eig_smem_per_warp(int NT) {
  // H (Householder vectors), Y (eigenvectors), v and q padded to NT + 4 for
  // float4 reads past the active size, d, e, e2, lam (NT floats), act
  return sizeof(float) * (2 * (size_t)NT * pitch_of(NT) + 2 * (NT + 4) + 4 * NT) +
         sizeof(int) * NT;
}

// Number of eigenvalues of the symmetric tridiagonal (d, e2 = e^2) below x
// (Sturm sequence of the LDL^T pivots; tiny pivots are replaced by -pivmin).
__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int m, float x,
                                           float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = q < 0.f;
  for (int i = 1; i < m; ++i) {
    q = d[i] - x - __fdividef(e2[i - 1], q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.f;
  }
  return cnt;
}

// Tridiagonal LU with partial pivoting of (T - lambda I) (rows swapped when the
// subdiagonal exceeds the pivot): U has diagonals u0, u1, u2; mult/piv hold
// the eliminations.  Solves overwrite y with (T - lambda I)^{-1} y.
struct TriLU {
  float u0[tbk::MAX_NT], u1[tbk::MAX_NT], u2[tbk::MAX_NT], mult[tbk::MAX_NT];
  unsigned long long piv;
};

__device__ __forceinline__ void trilu_factor(TriLU& f, const float* d, const float* e, int m,
                                             float lam, float tiny) {
  float cd = d[0] - lam, cs = m > 1 ? e[0] : 0.f, cs2 = 0.f;
  f.piv = 0ull;
  for (int i = 0; i + 1 < m; ++i) {
    const float sub = e[i], nd = d[i + 1] - lam, ns = (i + 2 < m) ? e[i + 1] : 0.f;
    if (fabsf(cd) >= fabsf(sub)) {
      const float piv = fabsf(cd) < tiny ? (cd < 0.f ? -tiny : tiny) : cd;
      const float l = sub / piv;
      f.u0[i] = piv; f.u1[i] = cs; f.u2[i] = cs2; f.mult[i] = l;
      cd = nd - l * cs;
      cs = ns - l * cs2;
      cs2 = 0.f;
    } else {
      const float l = cd / sub;
      f.u0[i] = sub; f.u1[i] = nd; f.u2[i] = ns; f.mult[i] = l;
      f.piv |= 1ull << i;
      cd = cs - l * nd;
      cs = cs2 - l * ns;
      cs2 = 0.f;
    }
  }
  f.u0[m - 1] = fabsf(cd) < tiny ? (cd < 0.f ? -tiny : tiny) : cd;
  f.u1[m - 1] = 0.f;
  f.u2[m - 1] = 0.f;
}

__device__ __forceinline__ void trilu_solve(const TriLU& f, float* y, int m) {
  for (int i = 0; i + 1 < m; ++i) {          // apply P and L^{-1}
    float a = y[i], b = y[i + 1];
    if ((f.piv >> i) & 1ull) { const float t = a; a = b; b = t; }
    y[i] = a;
    y[i + 1] = b - f.mult[i] * a;
  }
  for (int i = m - 1; i >= 0; --i) {         // U^{-1}
    float t = y[i];
    if (i + 1 < m) t -= f.u1[i] * y[i + 1];
    if (i + 2 < m) t -= f.u2[i] * y[i + 2];
    y[i] = t / f.u0[i];
  }
}

__global__ void __launch_bounds__(EW * 32) eig_tri_kernel(const EigArgs a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int NT = a.NT, PT = pitch_of(NT);
  unsigned char* base = smem + warp * eig_smem_per_warp(NT);
  float* H = reinterpret_cast<float*>(base);
  float* Y = H + NT * PT;
  float* vv = Y + NT * PT;
  float* qq = vv + NT + 4;
  float* d = qq + NT + 4;
  float* e = d + NT;
  float* e2 = e + NT;
  float* lam = e2 + NT;
  int* act = reinterpret_cast<int*>(lam + NT);
  const int i = blockIdx.x * EW + warp;
  if (i >= a.n) return;

  const unsigned long long mask = a.colmask[i];
  const int m = __popcll(mask);
  for (int x = lane; x < NT; x += 32)
    if ((mask >> x) & 1ull) act[__popcll(mask & ((1ull << x) - 1ull))] = x;
  __syncwarp();
  const double* Ti = a.T + (size_t)i * NT * NT;
  for (int x = 0; x < m; ++x)
    for (int y = lane; y < PT; y += 32)
      H[x * PT + y] = y < m ? (float)Ti[act[x] * NT + act[y]] : 0.f;
  for (int y = lane; y < NT + 4; y += 32) { vv[y] = 0.f; qq[y] = 0.f; }
  __syncwarp();

  // ---- Householder reduction to tridiagonal form.  Step j zeroes column j
  // below the subdiagonal with I - 2 v v^T (v supported on rows > j) and keeps
  // v in that column; lane owns rows x = lane, lane + 32.  Row updates run
  // over float4 chunks from the aligned chunk holding column j + 1 (the extra
  // columns get a zero update because v and q vanish there).
  for (int j = 0; j + 2 < m; ++j) {
    float xs = 0.f;
    for (int x = lane; x < m; x += 32)
      if (x > j) xs += H[x * PT + j] * H[x * PT + j];
    const float sig = tbk::warp_sum(xs);
    const float x0 = H[(j + 1) * PT + j];
    __syncwarp();
    if (sig - x0 * x0 <= 1e-30f * (sig + 1e-30f) || sig == 0.f) {
      if (lane == 0) e[j] = x0;
      for (int x = lane; x < m; x += 32)
        if (x > j) H[x * PT + j] = 0.f;      // identity reflection
      __syncwarp();
      continue;
    }
    const float alpha = x0 >= 0.f ? -sqrtf(sig) : sqrtf(sig);
    const float inv = rsqrtf(2.f * (sig - x0 * alpha));
    for (int x = lane; x < m; x += 32)
      vv[x] = x <= j ? 0.f : (x == j + 1 ? (x0 - alpha) : H[x * PT + j]) * inv;
    __syncwarp();
    const int c0 = (j + 1) & ~3;
    float kp = 0.f;
    for (int x = lane; x < m; x += 32) {
      float p = 0.f;
      if (x > j) {
        const float* row = H + x * PT;
        for (int l = c0; l < m; l += 4) {
          const float4 h4 = *reinterpret_cast<const float4*>(row + l);
          const float4 v4 = *reinterpret_cast<const float4*>(vv + l);
          p += h4.x * v4.x + h4.y * v4.y + h4.z * v4.z + h4.w * v4.w;
        }
      }
      qq[x] = p;
      kp += p * vv[x];
    }
    const float K = tbk::warp_sum(kp);
    __syncwarp();
    for (int x = lane; x < m; x += 32) qq[x] -= K * vv[x];
    __syncwarp();
    for (int x = lane; x < m; x += 32) {
      if (x > j) {
        const float vx = 2.f * vv[x], qx = 2.f * qq[x];
        float* row = H + x * PT;
        for (int l = c0; l < m; l += 4) {
          float4 h4 = *reinterpret_cast<float4*>(row + l);
          const float4 v4 = *reinterpret_cast<const float4*>(vv + l);
          const float4 q4 = *reinterpret_cast<const float4*>(qq + l);
          h4.x -= vx * q4.x + qx * v4.x;
          h4.y -= vx * q4.y + qx * v4.y;
          h4.z -= vx * q4.z + qx * v4.z;
          h4.w -= vx * q4.w + qx * v4.w;
          *reinterpret_cast<float4*>(row + l) = h4;
        }
      }
    }
    __syncwarp();
    for (int x = lane; x < m; x += 32)
      if (x > j) H[x * PT + j] = vv[x];      // keep v_j in column j
    if (lane == 0) e[j] = alpha;
    for (int x = lane; x < NT + 4; x += 32) { vv[x] = 0.f; qq[x] = 0.f; }
    __syncwarp();
  }
  for (int x = lane; x < m; x += 32) d[x] = H[x * PT + x];
  if (lane == 0) {
    if (m >= 2) e[m - 2] = H[(m - 1) * PT + (m - 2)];
    if (m >= 1) e[m - 1] = 0.f;
  }
  __syncwarp();
  float gl = 1e30f, gu = -1e30f, emax = 0.f;
  for (int x = lane; x < m; x += 32) {
    e2[x] = e[x] * e[x];
    const float rad = fabsf(e[x]) + (x > 0 ? fabsf(e[x - 1]) : 0.f);
    gl = fminf(gl, d[x] - rad);
    gu = fmaxf(gu, d[x] + rad);
    emax = fmaxf(emax, e[x] * e[x]);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gl = fminf(gl, __shfl_xor_sync(0xffffffffu, gl, o));
    gu = fmaxf(gu, __shfl_xor_sync(0xffffffffu, gu, o));
    emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
  __syncwarp();
  const float tnorm = fmaxf(fabsf(gl), fabsf(gu));
  const float pivmin = fmaxf(1e-30f, 1.2e-7f * 1.2e-7f * emax);
  gl -= 2.4e-7f * tnorm + pivmin;
  gu += 2.4e-7f * tnorm + pivmin;

  // ---- eigenvalues by bisection: lane owns indices k = lane and lane + 32
  {
    const int k0 = lane, k1 = lane + 32;
    float a0 = gl, b0 = gu, a1 = gl, b1 = gu;
    for (int it = 0; it < 64; ++it) {
      const bool go0 = k0 < m && (b0 - a0) > 2.4e-7f * fmaxf(fabsf(a0), fabsf(b0)) + pivmin;
      const bool go1 = k1 < m && (b1 - a1) > 2.4e-7f * fmaxf(fabsf(a1), fabsf(b1)) + pivmin;
      if (!__any_sync(0xffffffffu, go0 || go1)) break;
      const float m0 = 0.5f * (a0 + b0), m1 = 0.5f * (a1 + b1);
      if (go0) { if (sturm_count(d, e2, m, m0, pivmin) > k0) b0 = m0; else a0 = m0; }
      if (go1) { if (sturm_count(d, e2, m, m1, pivmin) > k1) b1 = m1; else a1 = m1; }
    }
    if (k0 < m) lam[k0] = 0.5f * (a0 + b0);
    if (k1 < m) lam[k1] = 0.5f * (a1 + b1);
  }
  __syncwarp();

  // ---- eigenvectors by inverse iteration (lane-parallel), Gram-Schmidt
  // inside clusters of close eigenvalues between iterations
  const float gtol = 1e-3f * tnorm;
  const float tiny = 1.2e-7f * tnorm + 1e-30f;
  for (int half = 0; half < 2; ++half) {
    const int k = lane + 32 * half;
    if (!__any_sync(0xffffffffu, k < m)) break;
    TriLU f;
    float y[tbk::MAX_NT];
    if (k < m) {
      trilu_factor(f, d, e, m, lam[k], tiny);
      for (int x = 0; x < m; ++x) y[x] = 1.f + 0.25f * (float)(((x * 7 + k * 13) % 17) - 8) / 8.f;
    }
    for (int it = 0; it < 3; ++it) {
      if (k < m) {
        trilu_solve(f, y, m);
        float nn = 0.f;
        for (int x = 0; x < m; ++x) nn += y[x] * y[x];
        const float s = rsqrtf(fmaxf(nn, 1e-30f));
        for (int x = 0; x < m; ++x) Y[x * PT + k] = y[x] * s;
      }
      __syncwarp();
      // clusters: runs of consecutive eigenvalues closer than gtol; members
      // are orthogonalised in index order against the earlier ones
      const int kb = 32 * half, ke = min(m, kb + 32);
      for (int kk = 1; kk < m; ++kk) {
        if (!(lam[kk] - lam[kk - 1] < gtol)) continue;
        if (kk < kb || kk >= ke) continue;
        int first = kk - 1;
        while (first > 0 && lam[first] - lam[first - 1] < gtol) --first;
        for (int kp2 = first; kp2 < kk; ++kp2) {
          float dt = 0.f;
          for (int x = lane; x < m; x += 32) dt += Y[x * PT + kk] * Y[x * PT + kp2];
          dt = tbk::warp_sum(dt);
          for (int x = lane; x < m; x += 32) Y[x * PT + kk] -= dt * Y[x * PT + kp2];
          __syncwarp();
        }
        float nn = 0.f;
        for (int x = lane; x < m; x += 32) nn += Y[x * PT + kk] * Y[x * PT + kk];
        nn = tbk::warp_sum(nn);
        const float s = rsqrtf(fmaxf(nn, 1e-30f));
        for (int x = lane; x < m; x += 32) Y[x * PT + kk] *= s;
        __syncwarp();
      }
      if (k < m)
        for (int x = 0; x < m; ++x) y[x] = Y[x * PT + k];
      __syncwarp();
    }
  }

  // ---- back-transformation: eigenvectors of T = H_0 ... H_{m-3} Y; lane
  // owns columns k = lane, lane + 32
  for (int j = m - 3; j >= 0; --j) {
    for (int k = lane; k < m; k += 32) {
      float t = 0.f;
      for (int x = j + 1; x < m; ++x) t += H[x * PT + j] * Y[x * PT + k];
      t *= 2.f;
      for (int x = j + 1; x < m; ++x) Y[x * PT + k] -= t * H[x * PT + j];
    }
  }
  __syncwarp();
  float* lf = a.lamf + (size_t)i * NT;
  float* zo = a.Zf + (size_t)i * NT * NT;
  for (int x = lane; x < m; x += 32) lf[x] = lam[x];
  for (int x = 0; x < m; ++x)
    for (int y = lane; y < m; y += 32) zo[x * NT + y] = Y[x * PT + y];
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
    b += sizeof(float) * NT * PT * 3;       // X, E, scratch
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
    // Loewdin orthonormalisation X <- X (I - E/2), E = X^T X - I (inverse
    // iteration leaves vectors of nearby eigenvalues orthogonal only to
    // ~eps ||T|| / gap), then FP64 Rayleigh quotients on the final vectors.
    float* Xf = reinterpret_cast<float*>(X);
    float* E = Xf + NT * PT;
    float* X2 = E + NT * PT;
    for (int q = tid; q < m * m; q += FT) {
      const int x = q / m, y = q - x * m;
      float t = 0.f;
      for (int l = 0; l < m; ++l) t += Xf[l * PT + x] * Xf[l * PT + y];
      E[x * PT + y] = 0.5f * (t - (x == y ? 1.f : 0.f));
    }
    __syncthreads();
    for (int q = tid; q < m * m; q += FT) {
      const int x = q / m, k = q - x * m;
      float t = Xf[x * PT + k];
      for (int l = 0; l < m; ++l) t -= Xf[x * PT + l] * E[l * PT + k];
      X2[x * PT + k] = t;
    }
    __syncthreads();
    for (int q = tid; q < m * m; q += FT) Xf[(q / m) * PT + q % m] = X2[(q / m) * PT + q % m];
    __syncthreads();
    const double* Ti = a.T + (size_t)i * NT * NT;
    for (int k = tid; k < m; k += FT) {
      double num = 0.0, den = 0.0;
      for (int x = 0; x < m; ++x) {
        double t = 0.0;
        for (int y = blo[x]; y < bhi[x]; ++y) t += Ti[act[x] * NT + act[y]] * (double)Xf[y * PT + k];
        num += (double)Xf[x * PT + k] * t;
        den += (double)Xf[x * PT + k] * (double)Xf[x * PT + k];
      }
      lam[k] = num / den;
    }
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
  c->eig_smem = EW * eig_smem_per_warp(NT);
  TB_CUDA_TRY(cudaFuncSetAttribute(eig_tri_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
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
  if (c->kry_fused && c->p.prec == TB_PREC_MIXED) return TB_OK;   // done in the Krylov kernel
  if (!c->kry_fused) {
    EigArgs ea{n, NT, c->T, c->colmask, c->Zf, c->lamf, kdim, c->d_status};
    eig_tri_kernel<<<(n + EW - 1) / EW, EW * 32, c->eig_smem, s>>>(ea);
    TB_CUDA_TRY(cudaGetLastError());
  }
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
