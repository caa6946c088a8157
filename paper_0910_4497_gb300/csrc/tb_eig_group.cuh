// The projected eigensolve of one target by a 64-thread group (two warps on
// their own named barrier), shared by the eigensolver kernel and the
// persistent Krylov + eigensolve kernel.  Steps (T' = the active part of the
// block tridiagonal T, m x m, m <= NT <= 64):
//     1. Householder reduction of T' to tridiagonal form, threads holding
//        rows in registers;
//     2. eigenvalues by Sturm-sequence bisection, threads owning eigenvalues;
//     3. eigenvectors from the twisted factorisation of T' - lambda I
//        (forward LDL^T and backward UDU^T pivots, twist index at the
//        smallest |gamma_r|, then the two bidiagonal recurrences), twice, the
//        second time at the tridiagonal Rayleigh quotient of the first vector;
//        Gram-Schmidt inside clusters of eigenvalues closer than 1e-3 ||T||,
//        and for a member that duplicates an earlier one (equal eigenvalues of
//        a split tridiagonal) inverse iteration with a pivoted LU from a fresh
//        start vector, the scheme of LAPACK's stein;
//     4. back-transformation through the stored reflections (compact WY
//        blocks of eight), threads holding columns in registers;
//   then, in the mixed path: 5. a first-order Loewdin step; 6. Rayleigh
//   quotients on the original block-tridiagonal T in double-float arithmetic;
//   7. ascending order, lambda, S and P = Y U; in the FP64 path the FP32
//   eigenpairs are written for the refinement kernel.
#pragma once
#include "tb_internal.cuh"

namespace {

struct XArgs {
  int n, NT;
  const double* T;
  const unsigned long long* colmask;
  const float* Y;                  // Krylov basis rows (mixed path)
  const int* h_off;
  float* Zf;                       // FP64 path: FP32 eigenvectors
  float* lamf;
  double* lambda;                  // mixed path: spectral record
  double* S;
  double* P;
  int* kdim;
  int* st;
};

// odd row pitch: lanes reading one column (rows x..x+31) or one row each
// (same column index) hit 32 different banks
__host__ __device__ inline int xpitch(int NT) { return NT + 1; }

// H holds the matrix, then E of the Loewdin step, then the band of T as FP32
// hi/lo pairs (12 columns per row), then staged rows of the Krylov basis
__host__ __device__ inline int epitch(int NT) { return NT + 4; }   // E rows 16-byte aligned

// register capacity of a row / column in the Householder and back-transform
// phases (a multiple of 16)
__host__ __device__ inline int ntc_of(int NT) { return NT <= 16 ? 16 : NT <= 32 ? 32 : NT <= 48 ? 48 : 64; }

// H also holds the reflections between the Householder and back-transform
// phases (NT - 2 rows of ntc_of(NT)), then the eigenvectors as rows (NT rows
// of ntc_of(NT)) in the Loewdin step
__host__ __device__ inline size_t xw_hsize(int NT) {
  const size_t a = (size_t)NT * epitch(NT), b = 24 * (size_t)NT;
  const size_t c = (size_t)NT * ntc_of(NT);
  const size_t ab = a > b ? a : b;
  return ab > c ? ab : c;
}

constexpr int GT = 64;             // threads per target (two warps)
constexpr int NSLICE = 2 * GT;     // spectrum-slicing points

// One scratch region serves, one phase at a time, the Householder vectors
// (4 ntc_of(NT) + 8 floats), the slicing counts (NSLICE) and the restart
// factorisation of the eigenvector phase (5 NT).
__host__ __device__ inline size_t xw_scratch(int NT) {
  size_t a = 5 * (size_t)NT, b = 4 * (size_t)ntc_of(NT) + 8;
  if (b > a) a = b;
  return a > (size_t)NSLICE ? a : (size_t)NSLICE;
}

__host__ __device__ inline size_t xw_smem_per_warp(int NT) {   // per target
  size_t b = sizeof(double) * NT;                          // lamd
  b += sizeof(float) * (xw_hsize(NT) + (size_t)NT * xpitch(NT) + 6 * (size_t)NT + xw_scratch(NT) + 8);
  b += sizeof(int) * 2 * NT;                               // act, rank
  return (b + 15) & ~size_t(15);
}

// The two warps of a target synchronise on their own named barrier.
struct Grp {
  int t;        // thread in the target's group, 0..63
  int wl;       // lane in its warp
  int gw;       // warp in the group
  int bid;      // named barrier id
  float* red;   // 8 floats of scratch
};

__device__ __forceinline__ void gsync(const Grp& g) {
  asm volatile("bar.sync %0, 64;" ::"r"(g.bid) : "memory");
}

__device__ __forceinline__ float gsum(const Grp& g, float v) {
  v = tbk::warp_sum(v);
  if (g.wl == 0) g.red[g.gw] = v;
  gsync(g);
  const float tot = g.red[0] + g.red[1];
  gsync(g);
  return tot;
}

// Sturm counts (number of eigenvalues below x) at two points at once: two
// independent dependency chains for the same thread.
__device__ __forceinline__ void sturm_count2(const float* d, const float* e2, int m, float xa,
                                             float xb, float pivmin, int& ca, int& cb) {
  float qa = d[0] - xa, qb = d[0] - xb;
  if (fabsf(qa) < pivmin) qa = -pivmin;
  if (fabsf(qb) < pivmin) qb = -pivmin;
  int na = qa < 0.f, nb = qb < 0.f;
  for (int i = 1; i < m; ++i) {
    const float di = d[i], ei = e2[i - 1];
    qa = di - xa - __fdividef(ei, qa);
    qb = di - xb - __fdividef(ei, qb);
    if (fabsf(qa) < pivmin) qa = -pivmin;
    if (fabsf(qb) < pivmin) qb = -pivmin;
    na += qa < 0.f;
    nb += qb < 0.f;
  }
  ca = na;
  cb = nb;
}

__device__ __forceinline__ float guard(float x, float tiny) {
  return fabsf(x) < tiny ? (x < 0.f ? -tiny : tiny) : x;
}

// Eigenvector of the tridiagonal (d, e) for the estimate lk from the twisted
// factorisation of T - lk I, written into column k of Y (pitch P): forward
// pivots Dp_i, backward pivots Dm_i, gamma_i = Dp_i + Dm_i - (d_i - lk), twist
// r = argmin |gamma|, z_r = 1, z_i = -(e_i / Dp_i) z_{i+1} (i < r),
// z_{i+1} = -(e_i / Dm_{i+1}) z_i (i >= r); normalised.  Only the output
// column is used as storage.
__device__ __forceinline__ void twisted_vector(const float* d, const float* e, const float* e2,
                                               int m, float lk, float tiny, float* Y, int P,
                                               int k) {
  float dp = guard(d[0] - lk, tiny);
  Y[k] = dp;
  for (int i = 1; i < m; ++i) {
    dp = guard((d[i] - lk) - __fdividef(e2[i - 1], dp), tiny);
    Y[i * P + k] = dp;
  }
  float dm = guard(d[m - 1] - lk, tiny);
  float best = fabsf(Y[(m - 1) * P + k]);
  int r = m - 1;
  for (int i = m - 2; i >= 0; --i) {
    const float di = d[i] - lk;
    dm = guard(di - __fdividef(e2[i], dm), tiny);
    const float g = fabsf(Y[i * P + k] + dm - di);
    if (g < best) { best = g; r = i; }
  }
  // U multipliers e_i / Dm_{i+1} for i = m-2 .. r, kept in rows i+1
  dm = guard(d[m - 1] - lk, tiny);
  for (int i = m - 2; i >= r; --i) {
    Y[(i + 1) * P + k] = __fdividef(e[i], dm);
    dm = guard((d[i] - lk) - __fdividef(e2[i], dm), tiny);
  }
  float nn = 1.f, z = 1.f;
  for (int i = r; i + 1 < m; ++i) {
    z = -Y[(i + 1) * P + k] * z;
    Y[(i + 1) * P + k] = z;
    nn += z * z;
  }
  z = 1.f;
  for (int i = r - 1; i >= 0; --i) {
    z = -__fdividef(e[i], Y[i * P + k]) * z;
    Y[i * P + k] = z;
    nn += z * z;
  }
  Y[r * P + k] = 1.f;
  const float sc = rsqrtf(nn);
  for (int i = 0; i < m; ++i) Y[i * P + k] *= sc;
}

// double-float accumulation: (hi, lo) += a * b for floats a, b (exact product)
__device__ __forceinline__ void df_fma(float& hi, float& lo, float a, float b) {
  const float p = a * b;
  const float pe = fmaf(a, b, -p);
  const float s = hi + p;
  const float bb = s - hi;
  const float err = (hi - (s - bb)) + (p - bb);
  hi = s;
  lo += err + pe;
}

// start vector of an inverse-iteration restart (deterministic, all components nonzero)
__device__ __forceinline__ float start_component(int x, int k) {
  unsigned h = (unsigned)x * 2654435761u ^ ((unsigned)k * 40503u + 0x9e3779b9u);
  h ^= h >> 13;
  h *= 0x5bd1e995u;
  h ^= h >> 15;
  return ((h & 1u) ? -1.f : 1.f) * (0.5f + (float)((h >> 1) & 1023u) * (1.0f / 1023.0f));
}

// Orthogonalise column c of Y against columns [c0, c) and normalise (whole
// group, one row per thread); returns the squared norm left after the
// projections.
__device__ __forceinline__ float orth_column(const Grp& g, float* Y, int P, int m, int c0, int c) {
  const int x = g.t;
  const bool hx = x < m;
  for (int c2 = c0; c2 < c; ++c2) {
    const float dt = gsum(g, hx ? Y[x * P + c] * Y[x * P + c2] : 0.f);
    if (hx) Y[x * P + c] -= dt * Y[x * P + c2];
  }
  const float nn = gsum(g, hx ? Y[x * P + c] * Y[x * P + c] : 0.f);
  const float sc = rsqrtf(fmaxf(nn, 1e-30f));
  if (hx) Y[x * P + c] *= sc;
  gsync(g);
  return nn;
}

// Inverse iteration for column c at eigenvalue lk with the pivoted
// tridiagonal LU of T - lk I (the dlagtf/dlagts scheme), restarted from a
// fixed start vector and kept orthogonal to columns [c0, c): used when the
// twisted vector of a degenerate eigenvalue duplicates an earlier one (a split
// tridiagonal).  The factorisation and the solves run on thread 0.
__device__ void restart_column(const Grp& g, const float* d, const float* e, int m, float lk,
                               float tiny, float* Y, int P, int c0, int c, float* f) {
  float* u0 = f;              // reciprocal pivots
  float* u1 = f + m;          // first super-diagonal of U
  float* u2 = f + 2 * m;      // second super-diagonal of U
  float* ml = f + 3 * m;      // multipliers
  float* pv = f + 4 * m;      // 1 where rows k, k+1 were interchanged
  if (g.t == 0) {
    float ak = d[0] - lk, bk = m > 1 ? e[0] : 0.f;
    for (int k = 0; k + 1 < m; ++k) {
      const float ck = e[k], ak1 = d[k + 1] - lk, bk1 = k + 2 < m ? e[k + 1] : 0.f;
      if (fabsf(ak) >= fabsf(ck)) {
        const float piv = guard(ak, tiny);
        const float mult = ck / piv;
        u0[k] = 1.f / piv; u1[k] = bk; u2[k] = 0.f; ml[k] = mult; pv[k] = 0.f;
        ak = ak1 - mult * bk;
        bk = bk1;
      } else {
        const float mult = ak / ck;
        u0[k] = 1.f / ck; u1[k] = ak1; u2[k] = bk1; ml[k] = mult; pv[k] = 1.f;
        ak = bk - mult * ak1;
        bk = -mult * bk1;
      }
    }
    u0[m - 1] = 1.f / guard(ak, tiny);
  }
  if (g.t < m) Y[g.t * P + c] = start_component(g.t, c);
  gsync(g);
  for (int it = 0; it < 3; ++it) {
    orth_column(g, Y, P, m, c0, c);
    if (g.t == 0) {
      float yk = Y[c];
      for (int k = 0; k + 1 < m; ++k) {
        const float yk1 = Y[(k + 1) * P + c];
        if (pv[k] == 0.f) { Y[k * P + c] = yk; yk = yk1 - ml[k] * yk; }
        else { Y[k * P + c] = yk1; yk = yk - ml[k] * yk1; }
      }
      Y[(m - 1) * P + c] = yk;
      float y1 = 0.f, y2 = 0.f;
      for (int k = m - 1; k >= 0; --k) {
        float y = Y[k * P + c];
        if (k + 1 < m) y -= u1[k] * y1;
        if (k + 2 < m) y -= u2[k] * y2;
        y *= u0[k];
        Y[k * P + c] = y;
        y2 = y1;
        y1 = y;
      }
    }
    gsync(g);
    // rescale before the next projection (sum of squares, not a maximum:
    // one group reduction)
    const float nn = gsum(g, g.t < m ? Y[g.t * P + c] * Y[g.t * P + c] : 0.f);
    if (g.t < m) Y[g.t * P + c] *= rsqrtf(fmaxf(nn, 1e-30f));
    gsync(g);
  }
  orth_column(g, Y, P, m, c0, c);
}

// The projected eigensolve of target i by one 64-thread group (g: its
// thread, lane, warp and named barrier; base: its xw_smem_per_warp(NT) bytes
// of shared memory).  T, Y and the column mask are read through L2 only
// (ld.global.cg): in the persistent Krylov + eigensolve kernel they were
// written by another SM during the same launch.
template <bool FULL, int NTC>
__device__ __forceinline__ void eig_group(const XArgs& a, int i, Grp g, unsigned char* base) {
  static_assert(NTC % 16 == 0 && NTC <= GT, "row capacity");
  const int t = g.t;
  const int NT = a.NT, P = xpitch(NT);
  double* lamd = reinterpret_cast<double*>(base);
  float* H = reinterpret_cast<float*>(lamd + NT);
  float* Y = H + xw_hsize(NT);
  float* d = Y + NT * P;
  float* e = d + NT;
  float* e2 = e + NT;
  float* lam = e2 + NT;
  float* v = lam + NT;
  float* q = v + NT;
  float* fs = q + NT;                          // scratch: Householder vectors, then
  float* slc = fs;                             // the slicing counts, then the restart
  g.red = fs + xw_scratch(NT);                 // factorisation; 8 floats of reductions
  int* act = reinterpret_cast<int*>(g.red + 8);
  int* rank = act + NT;

  const unsigned long long mask = __ldcg(a.colmask + i);
  const int m = __popcll(mask);
  if (t < NT && ((mask >> t) & 1ull)) act[__popcll(mask & ((1ull << t) - 1ull))] = t;
  gsync(g);
  // T is block tridiagonal, stored compactly (tc_index); entries outside
  // the block band are zero
  const double* Ti = a.T + (size_t)i * tc_doubles(NT / 4);
  auto tget = [&](int x, int y) -> double {
    const int q = tc_index(x, y);
    return q < 0 ? 0.0 : __ldcg(Ti + q);
  };
  if (t < m) {
    const int ay = act[t];
    for (int x = 0; x < m; ++x) H[x * P + t] = (float)tget(act[x], ay);
  }
  gsync(g);

  // ---- 1. Householder with the rows in registers: thread t holds row t of
  // the active matrix (pairs of columns, zero past m).  Step j: the owner of
  // row j has published it (symmetry: column j below the diagonal is row j
  // right of it); the reflection I - 2 v v^T maps it to (alpha, 0, ...);
  // p = A v, K = v^T p, and A <- A - 2 v p^T - 2 p v^T + 4 K v v^T on the rows
  // below j (the same matrix as A - 2 v q^T - 2 q v^T with q = p - K v, with
  // one group barrier less); the owner of row j+1 then publishes it.  Four
  // group barriers per step: the pivot row and the partial sums are double
  // buffered.  The vectors are read as 16-byte broadcasts; column blocks left
  // of j+1 are skipped eight at a time.  Reflection j is kept for the
  // back-transform in Vr[j][0..NTC).
  float* const rowb = fs;                        // 2 x NTC: the published row
  float* const vs = fs + 2 * NTC;                // NTC: v (zero outside j+1..m-1)
  float* const ps = fs + 3 * NTC;                // NTC: p = A v (zero outside j+1..m-1)
  float* const rb = fs + 4 * NTC;                // 2 x 4: warp partials, by step parity
  float* const Vr = H;
  float2 ar[NTC / 2];
#pragma unroll
  for (int k = 0; k < NTC / 2; ++k) {
    const int c = 2 * k;
    ar[k].x = (t < m && c < m) ? H[t * P + c] : 0.f;
    ar[k].y = (t < m && c + 1 < m) ? H[t * P + c + 1] : 0.f;
  }
  gsync(g);                                      // H is overwritten by Vr below
  auto publish = [&](float* dst) {
#pragma unroll
    for (int k = 0; k < NTC / 2; k += 2)
      *reinterpret_cast<float4*>(dst + 2 * k) = make_float4(ar[k].x, ar[k].y, ar[k + 1].x, ar[k + 1].y);
  };
  if (t == 0 && m > 2) publish(rowb);
  gsync(g);
  for (int j = 0; j + 2 < m; ++j) {
    const float* rowj = rowb + (j & 1) * NTC;
    float* const rbj = rb + (j & 1) * 4;
    const bool hx = t > j && t < m;
    const float xj = rowj[j + 1];
    const float hxj = hx ? rowj[t] : 0.f;
    {
      const float sw = tbk::warp_sum(hxj * hxj);
      if (g.wl == 0) rbj[g.gw] = sw;
    }
    gsync(g);
    const float sig = rbj[0] + rbj[1];
    float* const vrj = Vr + j * NTC;
    if (sig - xj * xj <= 1e-30f * (sig + 1e-30f) || sig == 0.f) {
      if (t == 0) e[j] = xj;                      // identity: nothing to reduce
      if (t < NTC) vrj[t] = 0.f;
      if (t == j + 1) publish(rowb + ((j + 1) & 1) * NTC);
      gsync(g);
      continue;
    }
    const float alpha = xj >= 0.f ? -sqrtf(sig) : sqrtf(sig);
    const float inv = rsqrtf(2.f * (sig - xj * alpha));
    const float vx = hx ? (t == j + 1 ? (xj - alpha) : hxj) * inv : 0.f;
    if (t < NTC) {
      vs[t] = vx;
      vrj[t] = vx;
    }
    gsync(g);
    float2 pa = make_float2(0.f, 0.f), pb = make_float2(0.f, 0.f);
#pragma unroll
    for (int k = 0; k < NTC / 2; k += 4) {
      if (2 * k + 7 > j) {                       // uniform: the block holds a column > j
        const float4 v0 = *reinterpret_cast<const float4*>(vs + 2 * k);
        const float4 v1 = *reinterpret_cast<const float4*>(vs + 2 * k + 4);
        pa = __ffma2_rn(ar[k], make_float2(v0.x, v0.y), pa);
        pb = __ffma2_rn(ar[k + 1], make_float2(v0.z, v0.w), pb);
        pa = __ffma2_rn(ar[k + 2], make_float2(v1.x, v1.y), pa);
        pb = __ffma2_rn(ar[k + 3], make_float2(v1.z, v1.w), pb);
      }
    }
    const float pr = hx ? (pa.x + pa.y) + (pb.x + pb.y) : 0.f;
    if (t < NTC) ps[t] = pr;
    {
      const float kw = tbk::warp_sum(pr * vx);
      if (g.wl == 0) rbj[2 + g.gw] = kw;
    }
    gsync(g);
    if (hx) {
      const float K = rbj[2] + rbj[3];
      const float2 mv = make_float2(-2.f * vx, -2.f * vx);
      const float cq = -(2.f * pr - 4.f * K * vx);
      const float2 mq = make_float2(cq, cq);
#pragma unroll
      for (int k = 0; k < NTC / 2; k += 4) {
        if (2 * k + 7 > j) {
          const float4 v0 = *reinterpret_cast<const float4*>(vs + 2 * k);
          const float4 v1 = *reinterpret_cast<const float4*>(vs + 2 * k + 4);
          const float4 q0 = *reinterpret_cast<const float4*>(ps + 2 * k);
          const float4 q1 = *reinterpret_cast<const float4*>(ps + 2 * k + 4);
          ar[k] = __ffma2_rn(mv, make_float2(q0.x, q0.y), __ffma2_rn(mq, make_float2(v0.x, v0.y), ar[k]));
          ar[k + 1] = __ffma2_rn(mv, make_float2(q0.z, q0.w), __ffma2_rn(mq, make_float2(v0.z, v0.w), ar[k + 1]));
          ar[k + 2] = __ffma2_rn(mv, make_float2(q1.x, q1.y), __ffma2_rn(mq, make_float2(v1.x, v1.y), ar[k + 2]));
          ar[k + 3] = __ffma2_rn(mv, make_float2(q1.z, q1.w), __ffma2_rn(mq, make_float2(v1.z, v1.w), ar[k + 3]));
        }
      }
    }
    if (t == 0) e[j] = alpha;
    if (t == j + 1) publish(rowb + ((j + 1) & 1) * NTC);
    gsync(g);
  }
  {
    // diagonal and last off-diagonal entry from the rows
    float dt = 0.f, et = 0.f;
#pragma unroll
    for (int k = 0; k < NTC / 2; ++k) {
      if (2 * k == t) dt = ar[k].x;
      if (2 * k + 1 == t) dt = ar[k].y;
      if (2 * k == m - 2) et = ar[k].x;
      if (2 * k + 1 == m - 2) et = ar[k].y;
    }
    if (t < m) d[t] = dt;
    if (t == m - 1 && m >= 2) e[m - 2] = et;
    if (t == 0) e[m - 1] = 0.f;
  }
  gsync(g);
  float lmin = 1e30f, lmax = -1e30f, emax = 0.f;
  if (t < m) {
    e2[t] = e[t] * e[t];
    const float rad = fabsf(e[t]) + (t > 0 ? fabsf(e[t - 1]) : 0.f);
    lmin = d[t] - rad;
    lmax = d[t] + rad;
    emax = e[t] * e[t];
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    lmin = fminf(lmin, __shfl_xor_sync(0xffffffffu, lmin, o));
    lmax = fmaxf(lmax, __shfl_xor_sync(0xffffffffu, lmax, o));
    emax = fmaxf(emax, __shfl_xor_sync(0xffffffffu, emax, o));
  }
  if (g.wl == 0) { g.red[3 * g.gw] = lmin; g.red[3 * g.gw + 1] = lmax; g.red[3 * g.gw + 2] = emax; }
  gsync(g);
  lmin = fminf(g.red[0], g.red[3]);
  lmax = fmaxf(g.red[1], g.red[4]);
  emax = fmaxf(g.red[2], g.red[5]);
  gsync(g);
  const float tnorm = fmaxf(fmaxf(fabsf(lmin), fabsf(lmax)), 1e-30f);
  const float pivmin = fmaxf(1e-30f, 1.2e-7f * 1.2e-7f * emax);
  const float tiny = 1.2e-7f * tnorm;
  lmin -= 2.4e-7f * tnorm + pivmin;
  lmax += 2.4e-7f * tnorm + pivmin;

  // ---- 2. eigenvalues: counts at NSLICE points splitting [lmin, lmax]
  // evenly (two per thread), then trisection from the slice holding each
  // eigenvalue (thread t owns eigenvalue t), a fixed number of rounds shrinking
  // the slice to 2.4e-7 ||T||
  {
    const float h = (lmax - lmin) / (float)(NSLICE + 1);
    int s0 = 0, s1 = 0;
    sturm_count2(d, e2, m, lmin + h * (float)(t + 1), lmin + h * (float)(t + 1 + GT), pivmin, s0,
                 s1);
    slc[t] = (float)s0;
    slc[t + GT] = (float)s1;
    gsync(g);
    float lo = lmin, hi = lmax;
    for (int u = 0; u < NSLICE; ++u) {            // point u + 1 has slc[u] eigenvalues below
      const float xu = lmin + h * (float)(u + 1);
      if ((int)slc[u] > t) hi = fminf(hi, xu); else lo = fmaxf(lo, xu);
    }
    const float tol = 2.4e-7f * tnorm + pivmin;
    const int rounds = (h > tol) ? (int)ceilf(logf(h / tol) * 0.91023922f) : 0;   // log_3
    if (t < m) {
      for (int it = 0; it < rounds; ++it) {
        const float w = (hi - lo) * (1.f / 3.f);
        const float p1 = lo + w, p2 = hi - w;
        int c1, c2;
        sturm_count2(d, e2, m, p1, p2, pivmin, c1, c2);
        if (c1 > t) hi = p1;
        else if (c2 > t) { lo = p1; hi = p2; }
        else lo = p2;
      }
      lam[t] = 0.5f * (lo + hi);
    }
  }
  gsync(g);
  // ---- 3. eigenvectors: twisted factorisations, twice (the second at the
  // tridiagonal Rayleigh quotient of the first vector, kept inside the
  // eigenvalue's own bracket so that a vector mixed with a close neighbour
  // cannot move the shift onto that neighbour)
  if (t < m) {
    const float lk = lam[t];
    twisted_vector(d, e, e2, m, lk, tiny, Y, P, t);
    float n0 = 0.f, n1 = 0.f, zp = 0.f;
    for (int x = 0; x < m; ++x) {
      const float z = Y[x * P + t];
      n0 += d[x] * z * z;
      if (x > 0) n1 += e[x - 1] * zp * z;
      zp = z;
    }
    const float hw = 1.2e-7f * tnorm + pivmin;
    twisted_vector(d, e, e2, m, fminf(fmaxf(n0 + 2.f * n1, lk - hw), lk + hw), tiny, Y, P, t);
  }
  gsync(g);
  // Gram-Schmidt inside clusters of close eigenvalues (index order); a member
  // that loses most of its norm duplicated an earlier one and is recomputed
  const float gtol = 1e-3f * tnorm;
  for (int c = 1; c < m; ++c) {
    if (!(lam[c] - lam[c - 1] < gtol)) continue;
    int first = c - 1;
    while (first > 0 && lam[first] - lam[first - 1] < gtol) --first;
    const float nn = orth_column(g, Y, P, m, first, c);
    if (nn < 0.25f) restart_column(g, d, e, m, lam[c], tiny, Y, P, first, c, fs);
  }

  // ---- 4. back-transformation U = H_0 ... H_{m-3} Y: thread t keeps column
  // t of U in registers (pairs of rows) and applies the reflections one at a
  // time, the last first: u <- u - 2 (v^T u) v (v read as 16-byte broadcasts,
  // rows <= j skipped eight at a time).  No barriers: each thread owns its
  // column, and a blocked (WY) form would save no arithmetic here.  The
  // column stays in registers through the Loewdin step and the spectral
  // record.
  float2 u[NTC / 2];
#pragma unroll
  for (int k = 0; k < NTC / 2; ++k) {
    u[k].x = (t < m && 2 * k < m) ? Y[(2 * k) * P + t] : 0.f;
    u[k].y = (t < m && 2 * k + 1 < m) ? Y[(2 * k + 1) * P + t] : 0.f;
  }
  if (t < m) {
    for (int j = m - 3; j >= 0; --j) {
      const float* vj = Vr + j * NTC;
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < NTC / 2; k += 4) {
        if (2 * k + 7 > j) {
          const float4 v0 = *reinterpret_cast<const float4*>(vj + 2 * k);
          const float4 v1 = *reinterpret_cast<const float4*>(vj + 2 * k + 4);
          a0 = __ffma2_rn(u[k], make_float2(v0.x, v0.y), a0);
          a1 = __ffma2_rn(u[k + 1], make_float2(v0.z, v0.w), a1);
          a0 = __ffma2_rn(u[k + 2], make_float2(v1.x, v1.y), a0);
          a1 = __ffma2_rn(u[k + 3], make_float2(v1.z, v1.w), a1);
        }
      }
      const float s2 = -2.f * ((a0.x + a0.y) + (a1.x + a1.y));
      const float2 ss = make_float2(s2, s2);
#pragma unroll
      for (int k = 0; k < NTC / 2; k += 4) {
        if (2 * k + 7 > j) {
          const float4 v0 = *reinterpret_cast<const float4*>(vj + 2 * k);
          const float4 v1 = *reinterpret_cast<const float4*>(vj + 2 * k + 4);
          u[k] = __ffma2_rn(ss, make_float2(v0.x, v0.y), u[k]);
          u[k + 1] = __ffma2_rn(ss, make_float2(v0.z, v0.w), u[k + 1]);
          u[k + 2] = __ffma2_rn(ss, make_float2(v1.x, v1.y), u[k + 2]);
          u[k + 3] = __ffma2_rn(ss, make_float2(v1.z, v1.w), u[k + 3]);
        }
      }
    }
  }
  gsync(g);                                      // every thread is done with Vr

  // ---- 5. Loewdin U <- U (I - E), E = (U^T U - I) / 2: the eigenvectors as
  // rows Ut (16-byte rows, read as broadcasts) in H, thread b forms column b
  // of E from its register column into Y's space, then updates its column
  // u_b <- u_b - sum_c u_c E[c][b] from the rows, and U returns to Y.
  float* const Ut = H;
  if (t < m) {
#pragma unroll
    for (int k = 0; k < NTC / 2; k += 2)
      *reinterpret_cast<float4*>(Ut + t * NTC + 2 * k) = make_float4(u[k].x, u[k].y, u[k + 1].x, u[k + 1].y);
  }
  gsync(g);
  float* const E = Y;
  if (t < m) {
    for (int c = 0; c < m; ++c) {
      const float* uc = Ut + c * NTC;
      float2 a0 = make_float2(0.f, 0.f), a1 = make_float2(0.f, 0.f);
#pragma unroll
      for (int k = 0; k < NTC / 2; k += 2) {
        if (2 * k < m) {
          const float4 v = *reinterpret_cast<const float4*>(uc + 2 * k);
          a0 = __ffma2_rn(u[k], make_float2(v.x, v.y), a0);
          a1 = __ffma2_rn(u[k + 1], make_float2(v.z, v.w), a1);
        }
      }
      E[c * P + t] = 0.5f * (((a0.x + a0.y) + (a1.x + a1.y)) - (c == t ? 1.f : 0.f));
    }
  }
  gsync(g);
  if (t < m) {
    for (int c = 0; c < m; ++c) {
      const float ec = -E[c * P + t];
      const float2 e2 = make_float2(ec, ec);
      const float* uc = Ut + c * NTC;
#pragma unroll
      for (int k = 0; k < NTC / 2; k += 2) {
        if (2 * k < m) {
          const float4 v = *reinterpret_cast<const float4*>(uc + 2 * k);
          u[k] = __ffma2_rn(e2, make_float2(v.x, v.y), u[k]);
          u[k + 1] = __ffma2_rn(e2, make_float2(v.z, v.w), u[k + 1]);
        }
      }
    }
  }
  gsync(g);                                      // E (in Y's space) is read
  if (t < m) {
#pragma unroll
    for (int k = 0; k < NTC / 2; ++k) {
      if (2 * k < m) Y[(2 * k) * P + t] = u[k].x;
      if (2 * k + 1 < m) Y[(2 * k + 1) * P + t] = u[k].y;
    }
  }
  gsync(g);

  if constexpr (!FULL) {
    float* lf = a.lamf + (size_t)i * NT;
    float* zo = a.Zf + (size_t)i * NT * NT;
    if (t < m) lf[t] = lam[t];
    for (int x = 0; x < m; ++x)
      if (t < m) zo[x * NT + t] = Y[x * P + t];
    if (t == 0) a.kdim[i] = m;
    return;
  } else {
    // ---- 6. Rayleigh quotients on the original block-tridiagonal T: row x
    // couples to the active columns of its own and the adjacent Krylov blocks
    // (band [blo, bhi) in active indices); T staged as FP32 hi/lo pairs.
    int* blo = reinterpret_cast<int*>(v);
    int* bhi = reinterpret_cast<int*>(q);
    float* Thi = H;                       // [x][12]
    float* Tlo = H + NT * 12;
    if (t < m) {
      const int x = t, bx = act[x] >> 2;
      int lo = x, hi = x + 1;
      while (lo > 0 && (act[lo - 1] >> 2) >= bx - 1) --lo;
      while (hi < m && (act[hi] >> 2) <= bx + 1) ++hi;
      blo[x] = lo;
      bhi[x] = hi;
      for (int w = 0; w < hi - lo; ++w) {
        const double tv = tget(act[x], act[lo + w]);
        const float th = (float)tv;
        Thi[x * 12 + w] = th;
        Tlo[x * 12 + w] = (float)(tv - (double)th);
      }
    }
    gsync(g);
    if (t < m) {
      const int k = t;
      float nh = 0.f, nl = 0.f, dh = 0.f, dl = 0.f;
      for (int x = 0; x < m; ++x) {
        const int l0 = blo[x], nw = bhi[x] - l0;
        float th = 0.f, tl = 0.f;
        for (int w = 0; w < nw; ++w) {
          const float u = Y[(l0 + w) * P + k];
          df_fma(th, tl, Thi[x * 12 + w], u);
          tl += Tlo[x * 12 + w] * u;
        }
        const float ux = Y[x * P + k];
        df_fma(nh, nl, ux, th);
        nl += ux * tl;
        df_fma(dh, dl, ux, ux);
      }
      const double lk = ((double)nh + (double)nl) / ((double)dh + (double)dl);
      lamd[k] = lk;
      if (!isfinite(lk)) tbk::set_status(a.st, TB_ERR_NONFINITE, i);
    }
    gsync(g);
    // ---- 7. ascending order (ties by index), spectral record
    if (t < m) {
      int rk = 0;
      const double lk = lamd[t];
      for (int c = 0; c < m; ++c) rk += (lamd[c] < lk) || (lamd[c] == lk && c < t);
      rank[t] = rk;
    }
    gsync(g);
    double* lo = a.lambda + (size_t)i * NT;
    double* So = a.S + (size_t)i * 4 * NT;
    if (t < NT) {
      if (t < m) lo[rank[t]] = lamd[t];
      else lo[t] = 0.0;
#pragma unroll
      for (int al = 0; al < 4; ++al) {
        if (t < m) So[al * NT + rank[t]] = (double)Y[al * P + t];
        else So[al * NT + t] = 0.0;
      }
    }
    // P = Y[rows, active] U: rows staged through H in chunks of RW rows
    const int deg = a.h_off[i + 1] - a.h_off[i];
    const size_t rbase = (size_t)(i + a.h_off[i]) * 4;
    const int nrows = 4 * (deg + 1);
    const int RW = (int)(xw_hsize(NT) / NT);
    float* Yr = H;
    for (int r0 = 0; r0 < nrows; r0 += RW) {
      const int nr = min(RW, nrows - r0);
      gsync(g);
      if (t >= m && t < NT)                    // past the active columns: zeros
        for (int rr = 0; rr < nr; ++rr) Yr[rr * NT + t] = 0.f;
      if (t < m) {
        const int ax = act[t];
        int rr = 0;
        for (; rr + 3 < nr; rr += 4) {        // four independent loads in flight
          const float y0 = __ldcg(a.Y + (rbase + r0 + rr) * NT + ax);
          const float y1 = __ldcg(a.Y + (rbase + r0 + rr + 1) * NT + ax);
          const float y2 = __ldcg(a.Y + (rbase + r0 + rr + 2) * NT + ax);
          const float y3 = __ldcg(a.Y + (rbase + r0 + rr + 3) * NT + ax);
          Yr[rr * NT + t] = y0;
          Yr[(rr + 1) * NT + t] = y1;
          Yr[(rr + 2) * NT + t] = y2;
          Yr[(rr + 3) * NT + t] = y3;
        }
        for (; rr < nr; ++rr) Yr[rr * NT + t] = __ldcg(a.Y + (rbase + r0 + rr) * NT + ax);
      }
      gsync(g);
      if (t < NT) {
        int rr = 0;
        for (; rr + 1 < nr; rr += 2) {          // two rows at a time
          double* p0 = a.P + (rbase + r0 + rr) * NT;
          double* p1 = p0 + NT;
          if (t < m) {
            // rows of the basis as 16-byte broadcasts against the register column
            const float* y0 = Yr + rr * NT;
            const float* y1 = y0 + NT;
            float2 s0 = make_float2(0.f, 0.f), s1 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NTC / 2; k += 2) {
              if (2 * k < m) {
                const float4 v0 = *reinterpret_cast<const float4*>(y0 + 2 * k);
                const float4 v1 = *reinterpret_cast<const float4*>(y1 + 2 * k);
                s0 = __ffma2_rn(u[k], make_float2(v0.x, v0.y), s0);
                s0 = __ffma2_rn(u[k + 1], make_float2(v0.z, v0.w), s0);
                s1 = __ffma2_rn(u[k], make_float2(v1.x, v1.y), s1);
                s1 = __ffma2_rn(u[k + 1], make_float2(v1.z, v1.w), s1);
              }
            }
            p0[rank[t]] = (double)(s0.x + s0.y);
            p1[rank[t]] = (double)(s1.x + s1.y);
          } else {
            p0[t] = 0.0;
            p1[t] = 0.0;
          }
        }
        if (rr < nr) {
          double* p0 = a.P + (rbase + r0 + rr) * NT;
          if (t < m) {
            const float* y0 = Yr + rr * NT;
            float2 s0 = make_float2(0.f, 0.f);
#pragma unroll
            for (int k = 0; k < NTC / 2; k += 2) {
              if (2 * k < m) {
                const float4 v0 = *reinterpret_cast<const float4*>(y0 + 2 * k);
                s0 = __ffma2_rn(u[k], make_float2(v0.x, v0.y), s0);
                s0 = __ffma2_rn(u[k + 1], make_float2(v0.z, v0.w), s0);
              }
            }
            p0[rank[t]] = (double)(s0.x + s0.y);
          } else {
            p0[t] = 0.0;
          }
        }
      }
    }
    if (t == 0) a.kdim[i] = m;
  }
}

}  // namespace
