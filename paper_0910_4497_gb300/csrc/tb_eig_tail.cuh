// The projected eigensolve inside the block-Lanczos CTA: FP32 eigenpairs of the projected
// matrix T of one target (Sec. 3: the small Lanczos matrix is diagonalised by
// a dense symmetric eigensolver) computed by the whole CTA in shared memory
// that the Krylov basis no longer needs, followed (mixed path) by the spectral
// record lambda, S = U[seed rows], P = Y U.
//
// Steps (m = number of active Krylov columns, T_a = T restricted to them):
//   1. Householder reduction of T_a to tridiagonal (d, e), reflection vectors
//      kept in the columns they annihilate;
//   2. eigenvalues by Sturm-sequence multisection: four threads per
//      eigenvalue evaluate four interior points of its bracket per round;
//   3. eigenvectors of the tridiagonal matrix by inverse iteration, one thread
//      per eigenvalue (LU with partial pivoting of T - lambda I, pivots kept
//      as reciprocals, three solves), with Gram-Schmidt inside clusters of eigenvalues closer than
//      1e-3 ||T|| after every solve (the scheme of LAPACK's stein);
//   4. back-transformation U = H_0 H_1 ... H_{m-3} Y, then a first-order
//      Loewdin step that makes U orthonormal to FP32 rounding;
//   5. FP64 Rayleigh quotients u^T T u of the final vectors.
#pragma once
#include "tb_internal.cuh"

namespace tbtail {

__host__ __device__ inline int tpitch(int NT) { return NT + 4; }

// floats of shared workspace the tail needs for block order r (NT = 4r)
__host__ __device__ inline size_t tail_floats(int NT) {
  const size_t PT = tpitch(NT);
  return 2 * (size_t)NT * PT            // H, U
         + 5 * (size_t)NT * NT          // LU factors (u0, u1, u2, mult) and iterates
         + 2 * (size_t)(NT + 4)         // v, q
         + 7 * (size_t)NT               // d, e, e2, lam, act, piv (2 words)
         + 64;                          // reduction scratch
}

template <int NTH>
__device__ __forceinline__ float block_sum1(float v, float* red) {
  v = tbk::warp_sum(v);
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  __syncthreads();
  if (lane == 0) red[warp] = v;
  __syncthreads();
  float s = 0.f;
#pragma unroll
  for (int w = 0; w < NTH / 32; ++w) s += red[w];
  return s;
}

struct TailOut {
  float* lam;     // [NT] FP32 eigenvalues (ascending), shared
  float* U;       // [NT][tpitch] eigenvectors (columns), shared
  int* act;       // [NT] active column -> Krylov column
  int m;
  double* rq;     // [NT][2] FP64 Rayleigh quotient numerator, denominator
};

// Eigen-decomposition of the active part of T (FP64, global, NT x NT) in the
// shared workspace `ws`.  Every thread of the CTA must call it.
template <int NTH>
__device__ TailOut eig_tail(const double* __restrict__ Ti, unsigned long long mask, int NT,
                            float* ws, int* st, int target) {
  const int tid = threadIdx.x, lane = tid & 31;
  const int PT = tpitch(NT);
  float* H = ws;
  float* U = H + NT * PT;
  float* u0 = U + NT * PT;
  float* u1 = u0 + NT * NT;
  float* u2 = u1 + NT * NT;
  float* ml = u2 + NT * NT;
  float* Yv = ml + NT * NT;
  float* vv = Yv + NT * NT;
  float* qq = vv + NT + 4;
  float* d = qq + NT + 4;
  float* e = d + NT;
  float* e2 = e + NT;
  float* lam = e2 + NT;
  int* act = reinterpret_cast<int*>(lam + NT);
  unsigned* piv = reinterpret_cast<unsigned*>(act + NT);   // row swaps: words k, NT + k
  float* red = reinterpret_cast<float*>(piv + 2 * NT);
  const int m = __popcll(mask);
  for (int x = tid; x < NT; x += NTH)
    if ((mask >> x) & 1ull) act[__popcll(mask & ((1ull << x) - 1ull))] = x;
  for (int x = tid; x < NT + 4; x += NTH) { vv[x] = 0.f; qq[x] = 0.f; }
  __syncthreads();
  for (int q = tid; q < m * PT; q += NTH) {
    const int x = q / PT, y = q - x * PT;
    H[q] = y < m ? (float)Ti[act[x] * NT + act[y]] : 0.f;
  }
  __syncthreads();

  // ---- 1. Householder tridiagonalisation
  for (int j = 0; j + 2 < m; ++j) {
    // column norm and reflection vector (warp 0)
    if (tid < 32) {
      float xs = 0.f;
      for (int x = lane; x < m; x += 32)
        if (x > j) xs += H[x * PT + j] * H[x * PT + j];
      const float sig = tbk::warp_sum(xs);
      const float x0 = H[(j + 1) * PT + j];
      const bool skip = sig - x0 * x0 <= 1e-30f * (sig + 1e-30f) || sig == 0.f;
      const float alpha = skip ? x0 : (x0 >= 0.f ? -sqrtf(sig) : sqrtf(sig));
      const float inv = skip ? 0.f : rsqrtf(2.f * (sig - x0 * alpha));
      for (int x = lane; x < NT + 4; x += 32)     // whole vector: zeros outside (j, m)
        vv[x] = (x <= j || x >= m) ? 0.f : (x == j + 1 ? (x0 - alpha) : H[x * PT + j]) * inv;
      if (lane == 0) e[j] = alpha;
    }
    __syncthreads();
    // p = A' v, four threads per row
    const int c0 = (j + 1) & ~3;
    {
      const int x = tid >> 2, part = tid & 3;
      float p = 0.f;
      if (x > j && x < m) {
        const float* row = H + x * PT;
        for (int l = c0 + 4 * part; l < m; l += 16) {
          const float4 h4 = *reinterpret_cast<const float4*>(row + l);
          const float4 v4 = *reinterpret_cast<const float4*>(vv + l);
          p += h4.x * v4.x + h4.y * v4.y + h4.z * v4.z + h4.w * v4.w;
        }
      }
      p += __shfl_xor_sync(0xffffffffu, p, 1);
      p += __shfl_xor_sync(0xffffffffu, p, 2);
      if (part == 0 && x < NT) qq[x] = (x > j && x < m) ? p : 0.f;
    }
    __syncthreads();
    // K = v.p, reduced by every warp for itself (no block barrier)
    float kp = 0.f;
    for (int x = lane; x < m; x += 32) kp += qq[x] * vv[x];
    const float K = tbk::warp_sum(kp);
    // rank-2 update A' -= 2 (v q^T + q v^T), q = p - K v, over float4 chunks
    // starting at the chunk that holds column j; column j receives v_j
    {
      const int cj = j & ~3;
      const int nch = (m - cj + 3) >> 2;
      for (int q = tid; q < (m - j - 1) * nch; q += NTH) {
        const int x = j + 1 + q / nch, l = cj + 4 * (q % nch);
        float4 h4 = *reinterpret_cast<float4*>(H + x * PT + l);
        const float4 v4 = *reinterpret_cast<const float4*>(vv + l);
        float4 q4 = *reinterpret_cast<const float4*>(qq + l);
        q4.x -= K * v4.x; q4.y -= K * v4.y; q4.z -= K * v4.z; q4.w -= K * v4.w;
        const float vxr = vv[x];
        const float vx = 2.f * vxr, qx = 2.f * (qq[x] - K * vxr);
        h4.x -= vx * q4.x + qx * v4.x;
        h4.y -= vx * q4.y + qx * v4.y;
        h4.z -= vx * q4.z + qx * v4.z;
        h4.w -= vx * q4.w + qx * v4.w;
        if (l <= j && j < l + 4) {
          const int cc = j - l;
          if (cc == 0) h4.x = vxr; else if (cc == 1) h4.y = vxr; else if (cc == 2) h4.z = vxr; else h4.w = vxr;
        }
        *reinterpret_cast<float4*>(H + x * PT + l) = h4;
      }
    }
    __syncthreads();
  }
  __syncthreads();
  for (int x = tid; x < m; x += NTH) d[x] = H[x * PT + x];
  if (tid == 0) {
    if (m >= 2) e[m - 2] = H[(m - 1) * PT + (m - 2)];
    if (m >= 1) e[m - 1] = 0.f;
  }
  __syncthreads();
  // Gershgorin interval, pivot floor
  float gl = 1e30f, gu = -1e30f, emax = 0.f;
  if (tid < 32) {
    for (int x = lane; x < m; x += 32) {
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
    if (lane == 0) { red[0] = gl; red[1] = gu; red[2] = emax; }
  }
  for (int x = tid; x < m; x += NTH) e2[x] = e[x] * e[x];
  __syncthreads();
  gl = red[0];
  gu = red[1];
  emax = red[2];
  const float tnorm = fmaxf(fabsf(gl), fabsf(gu));
  const float pivmin = fmaxf(1e-30f, 1.2e-7f * 1.2e-7f * emax);
  gl -= 2.4e-7f * tnorm + pivmin;
  gu += 2.4e-7f * tnorm + pivmin;

  // ---- 2. eigenvalues: multisection, four threads per eigenvalue
  for (int base = 0; base < m; base += NTH / 4) {
    const int k = base + (tid >> 2), part = tid & 3;
    float a = gl, b = gu;
    for (int it = 0; it < 40; ++it) {
      const bool go = k < m && (b - a) > 2.4e-7f * fmaxf(fabsf(a), fabsf(b)) + pivmin;
      if (!__syncthreads_or(go)) break;
      const float h = (b - a) * 0.2f;
      const float xq = a + h * (float)(part + 1);
      int cnt = 0;
      if (go) {
        float q = d[0] - xq;
        if (fabsf(q) < pivmin) q = -pivmin;
        cnt = q < 0.f;
        for (int ii = 1; ii < m; ++ii) {
          q = d[ii] - xq - __fdividef(e2[ii - 1], q);
          if (fabsf(q) < pivmin) q = -pivmin;
          cnt += q < 0.f;
        }
      }
      // counts of the group's four points; new bracket between the last point
      // with count <= k and the first with count > k
      const int gbase = lane & ~3;
      float na = a, nb = b;
      bool found = false;
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        const int cu = __shfl_sync(0xffffffffu, cnt, gbase + u);
        const float xu = a + h * (float)(u + 1);
        if (!found) {
          if (cu > k) { nb = xu; found = true; } else { na = xu; }
        }
      }
      if (go) { a = na; b = nb; }
    }
    if (part == 0 && k < m) lam[k] = 0.5f * (a + b);
  }
  __syncthreads();

  // ---- 3. eigenvectors of the tridiagonal matrix by inverse iteration
  const float gtol = 1e-3f * tnorm;
  const float tiny = 1.2e-7f * tnorm + 1e-30f;
  for (int k = tid; k < m; k += NTH) {
    const float lk = lam[k];
    float cd = d[0] - lk, cs = m > 1 ? e[0] : 0.f, cs2 = 0.f;
    unsigned pv0 = 0u, pv1 = 0u;
    for (int ii = 0; ii + 1 < m; ++ii) {
      const float sub = e[ii], nd = d[ii + 1] - lk, ns = (ii + 2 < m) ? e[ii + 1] : 0.f;
      if (fabsf(cd) >= fabsf(sub)) {
        const float pvt = fabsf(cd) < tiny ? (cd < 0.f ? -tiny : tiny) : cd;
        const float rp = __frcp_rn(pvt);
        const float l = sub * rp;
        u0[ii * NT + k] = rp; u1[ii * NT + k] = cs; u2[ii * NT + k] = cs2; ml[ii * NT + k] = l;
        cd = nd - l * cs;
        cs = ns - l * cs2;
      } else {
        const float rp = __frcp_rn(sub);
        const float l = cd * rp;
        u0[ii * NT + k] = rp; u1[ii * NT + k] = nd; u2[ii * NT + k] = ns; ml[ii * NT + k] = l;
        if (ii < 32) pv0 |= 1u << ii; else pv1 |= 1u << (ii - 32);
        cd = cs - l * nd;
        cs = cs2 - l * ns;
      }
      cs2 = 0.f;
    }
    u0[(m - 1) * NT + k] = __frcp_rn(fabsf(cd) < tiny ? (cd < 0.f ? -tiny : tiny) : cd);
    u1[(m - 1) * NT + k] = 0.f;
    u2[(m - 1) * NT + k] = 0.f;
    if (m >= 2) u2[(m - 2) * NT + k] = 0.f;
    piv[k] = pv0;
    piv[NT + k] = pv1;
    for (int x = 0; x < m; ++x)
      Yv[x * NT + k] = 1.f + 0.25f * (float)(((x * 7 + k * 13) % 17) - 8) / 8.f;
  }
  __syncthreads();
  for (int it = 0; it < 3; ++it) {
    for (int k = tid; k < m; k += NTH) {
      const unsigned pv0 = piv[k], pv1 = piv[NT + k];
      for (int ii = 0; ii + 1 < m; ++ii) {
        float a0 = Yv[ii * NT + k], b0 = Yv[(ii + 1) * NT + k];
        const bool sw = ii < 32 ? ((pv0 >> ii) & 1u) : ((pv1 >> (ii - 32)) & 1u);
        if (sw) { const float t = a0; a0 = b0; b0 = t; }
        Yv[ii * NT + k] = a0;
        Yv[(ii + 1) * NT + k] = b0 - ml[ii * NT + k] * a0;
      }
      float y1 = 0.f, y2 = 0.f, nn = 0.f;
      for (int ii = m - 1; ii >= 0; --ii) {
        const float t = (Yv[ii * NT + k] - u1[ii * NT + k] * y1 - u2[ii * NT + k] * y2) * u0[ii * NT + k];
        Yv[ii * NT + k] = t;
        y2 = y1;
        y1 = t;
        nn += t * t;
      }
      const float s = rsqrtf(fmaxf(nn, 1e-30f));
      for (int ii = 0; ii < m; ++ii) Yv[ii * NT + k] *= s;
    }
    __syncthreads();
    // Gram-Schmidt inside clusters (warp 0; lanes over components)
    if (tid < 32) {
      for (int kk = 1; kk < m; ++kk) {
        if (!(lam[kk] - lam[kk - 1] < gtol)) continue;
        int first = kk - 1;
        while (first > 0 && lam[first] - lam[first - 1] < gtol) --first;
        for (int k2 = first; k2 < kk; ++k2) {
          float dt = 0.f;
          for (int x = lane; x < m; x += 32) dt += Yv[x * NT + kk] * Yv[x * NT + k2];
          dt = tbk::warp_sum(dt);
          for (int x = lane; x < m; x += 32) Yv[x * NT + kk] -= dt * Yv[x * NT + k2];
          __syncwarp();
        }
        float nn = 0.f;
        for (int x = lane; x < m; x += 32) nn += Yv[x * NT + kk] * Yv[x * NT + kk];
        nn = tbk::warp_sum(nn);
        const float s = rsqrtf(fmaxf(nn, 1e-30f));
        for (int x = lane; x < m; x += 32) Yv[x * NT + kk] *= s;
        __syncwarp();
      }
    }
    __syncthreads();
  }

  // ---- 4. back-transformation U = H_0 ... H_{m-3} Y (U starts as Y)
  for (int q = tid; q < m * m; q += NTH) {
    const int x = q / m, k = q - x * m;
    U[x * PT + k] = Yv[x * NT + k];
  }
  __syncthreads();
  float* tk = Yv;   // reuse: per-column dot products
  for (int j = m - 3; j >= 0; --j) {
    {
      const int k = tid >> 2, part = tid & 3;
      float t = 0.f;
      if (k < m)
        for (int x = j + 1 + part; x < m; x += 4) t += H[x * PT + j] * U[x * PT + k];
      t += __shfl_xor_sync(0xffffffffu, t, 1);
      t += __shfl_xor_sync(0xffffffffu, t, 2);
      if (part == 0 && k < m) tk[k] = 2.f * t;
    }
    __syncthreads();
    for (int q = tid; q < (m - j - 1) * m; q += NTH) {
      const int x = j + 1 + q / m, k = q % m;
      U[x * PT + k] -= tk[k] * H[x * PT + j];
    }
    __syncthreads();
  }
  // ---- 4b. Loewdin orthonormalisation U <- U (I - E/2), E = U^T U - I.
  // Inverse-iteration vectors of eigenvalues a little apart are orthogonal
  // only to ~eps ||T|| / gap; the density matrix is sensitive to that, not
  // to rotations inside an orthonormal set.  Error after the step: O(|E|^2).
  {
    float* E = u1;                          // [m][m]
    for (int q = tid; q < m * m; q += NTH) {
      const int x = q / m, y = q - x * m;
      float t = 0.f;
      for (int l = 0; l < m; ++l) t += U[l * PT + x] * U[l * PT + y];
      E[q] = 0.5f * (t - (x == y ? 1.f : 0.f));
    }
    __syncthreads();
    for (int q = tid; q < m * m; q += NTH) {
      const int x = q / m, k = q - x * m;
      float t = U[x * PT + k];
      for (int l = 0; l < m; ++l) t -= U[x * PT + l] * E[l * m + k];
      Yv[x * NT + k] = t;
    }
    __syncthreads();
    for (int q = tid; q < m * m; q += NTH) {
      const int x = q / m, k = q - x * m;
      U[x * PT + k] = Yv[x * NT + k];
    }
    __syncthreads();
  }

  // ---- 5. FP64 Rayleigh quotients lam_k = u_k^T T u_k / u_k^T u_k.  T_a is
  // block tridiagonal in the Krylov block index, so row x couples only to
  // active columns of the adjacent blocks; the FP32 tridiagonalisation left
  // eigenvalue errors of order m eps ||T||, the quotient is accurate to the
  // square of the eigenvector error.
  {
    double* rq = reinterpret_cast<double*>(u0);        // [m][2] partial sums
    double* Tsh = reinterpret_cast<double*>(u1);       // [m][m] active T (u1, u2 free now)
    int* blo = reinterpret_cast<int*>(ml);             // band of row x: [blo, bhi)
    int* bhi = blo + NT;
    for (int q = tid; q < m * m; q += NTH) {
      const int x = q / m, y = q - x * m;
      Tsh[q] = Ti[act[x] * NT + act[y]];
    }
    for (int x = tid; x < m; x += NTH) {
      const int bx = act[x] >> 2;
      int lo = x, hi = x + 1;
      while (lo > 0 && (act[lo - 1] >> 2) >= bx - 1) --lo;
      while (hi < m && (act[hi] >> 2) <= bx + 1) ++hi;
      blo[x] = lo;
      bhi[x] = hi;
    }
    __syncthreads();
    static_assert(NTH / 4 >= tbk::MAX_NT, "one pass of four threads per eigenvector");
    {
      const int k = tid >> 2, part = tid & 3;
      double num = 0.0, den = 0.0;
      for (int x = part; x < m && k < m; x += 4) {
        const double ux = (double)U[x * PT + k];
        double t = 0.0;
        for (int y = blo[x]; y < bhi[x]; ++y) t += Tsh[x * m + y] * (double)U[y * PT + k];
        num += ux * t;
        den += ux * ux;
      }
      num += __shfl_xor_sync(0xffffffffu, num, 1);
      num += __shfl_xor_sync(0xffffffffu, num, 2);
      den += __shfl_xor_sync(0xffffffffu, den, 1);
      den += __shfl_xor_sync(0xffffffffu, den, 2);
      if (part == 0 && k < m) { rq[2 * k] = num; rq[2 * k + 1] = den; }
    }
    __syncthreads();
  }
  (void)st;
  (void)target;
  return TailOut{lam, U, act, m, reinterpret_cast<double*>(u0)};
}

}  // namespace tbtail
