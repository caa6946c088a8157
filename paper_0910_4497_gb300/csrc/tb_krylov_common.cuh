// Helpers shared by the per-target and the grouped block-Lanczos kernels:
// 4-wide vector loads and stores, and the 4x4 Cholesky factor and triangular
// inverse of the in-block QR (Cholesky QR of the Gram matrix W^T W = R^T R).
#pragma once
#include "tb_internal.cuh"

namespace tbkry {

template <typename TV>
struct alignas(4 * sizeof(TV)) vec4 {
  TV v[4];
};

template <typename TV>
__device__ __forceinline__ vec4<TV> ld4(const TV* p) {
  return *reinterpret_cast<const vec4<TV>*>(p);
}
template <typename TV>
__device__ __forceinline__ void st4(TV* p, const vec4<TV>& x) {
  *reinterpret_cast<vec4<TV>*>(p) = x;
}
template <typename TV>
__device__ __forceinline__ vec4<TV> ldg4(const TV* p) {
  vec4<TV> r;
  if constexpr (sizeof(TV) == 4) {
    float4 t = __ldg(reinterpret_cast<const float4*>(p));
    r.v[0] = t.x; r.v[1] = t.y; r.v[2] = t.z; r.v[3] = t.w;
  } else {
    double2 t0 = __ldg(reinterpret_cast<const double2*>(p));
    double2 t1 = __ldg(reinterpret_cast<const double2*>(p) + 1);
    r.v[0] = t0.x; r.v[1] = t0.y; r.v[2] = t1.x; r.v[3] = t1.y;
  }
  return r;
}

// Cholesky of a 4x4 Gram matrix g (row-major) into the upper-triangular R
// (row-major); returns false when a pivot is not a healthy fraction of its
// diagonal or falls near the deflation threshold.
// `well` reports whether every pivot keeps at least a quarter of its diagonal
// (then kappa(W)^2 <= ~16 and one Cholesky-QR pass is orthogonal to ~16 eps).
template <typename TV>
__device__ __forceinline__ bool chol4(const TV (&g)[16], TV (&R)[16], TV rel, double abs_tol,
                                      bool& well) {
#pragma unroll
  for (int q = 0; q < 16; ++q) R[q] = (TV)0;
  bool ok = true;
  well = true;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    TV d = g[c * 4 + c];
#pragma unroll
    for (int j = 0; j < c; ++j) d -= R[j * 4 + c] * R[j * 4 + c];
    if (!(d > rel * g[c * 4 + c]) || !(d > (TV)(abs_tol * abs_tol))) ok = false;
    if (!(d >= (TV)0.25 * g[c * 4 + c])) well = false;
    const TV dd = d > (TV)0 ? d : (TV)1;
    const TV inv = (TV)rsqrt(dd);
    const TV rc = dd * inv;
    R[c * 4 + c] = rc;
#pragma unroll
    for (int e = c + 1; e < 4; ++e) {
      TV t = g[c * 4 + e];
#pragma unroll
      for (int j = 0; j < c; ++j) t -= R[j * 4 + c] * R[j * 4 + e];
      R[c * 4 + e] = t * inv;
    }
  }
  return ok;
}

// The same factorisation, also returning the reciprocal pivots 1/R[c][c] (the
// reciprocal square roots the factorisation forms anyway).
template <typename TV>
__device__ __forceinline__ bool chol4(const TV (&g)[16], TV (&R)[16], TV rel, double abs_tol,
                                      bool& well, TV (&dinv)[4]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) R[q] = (TV)0;
  bool ok = true;
  well = true;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    TV d = g[c * 4 + c];
#pragma unroll
    for (int j = 0; j < c; ++j) d -= R[j * 4 + c] * R[j * 4 + c];
    if (!(d > rel * g[c * 4 + c]) || !(d > (TV)(abs_tol * abs_tol))) ok = false;
    if (!(d >= (TV)0.25 * g[c * 4 + c])) well = false;
    const TV dd = d > (TV)0 ? d : (TV)1;
    const TV inv = (TV)rsqrt(dd);
    dinv[c] = inv;
    R[c * 4 + c] = dd * inv;
#pragma unroll
    for (int e = c + 1; e < 4; ++e) {
      TV t = g[c * 4 + e];
#pragma unroll
      for (int j = 0; j < c; ++j) t -= R[j * 4 + c] * R[j * 4 + e];
      R[c * 4 + e] = t * inv;
    }
  }
  return ok;
}

// Inverse of an upper-triangular 4x4 R from its reciprocal pivots (no division).
template <typename TV>
__device__ __forceinline__ void triinv4(const TV (&R)[16], const TV (&dinv)[4], TV (&X)[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) X[q] = (TV)0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    X[c * 4 + c] = dinv[c];
#pragma unroll
    for (int rr = c - 1; rr >= 0; --rr) {
      TV t = (TV)0;
#pragma unroll
      for (int j = rr + 1; j <= c; ++j) t += R[rr * 4 + j] * X[j * 4 + c];
      X[rr * 4 + c] = -t * dinv[rr];
    }
  }
}

// Inverse of an upper-triangular 4x4 R (row-major).
template <typename TV>
__device__ __forceinline__ void triinv4(const TV (&R)[16], TV (&X)[16]) {
#pragma unroll
  for (int q = 0; q < 16; ++q) X[q] = (TV)0;
#pragma unroll
  for (int c = 0; c < 4; ++c) {
    X[c * 4 + c] = (TV)1 / R[c * 4 + c];
#pragma unroll
    for (int rr = c - 1; rr >= 0; --rr) {
      TV t = (TV)0;
#pragma unroll
      for (int j = rr + 1; j <= c; ++j) t += R[rr * 4 + j] * X[j * 4 + c];
      X[rr * 4 + c] = -t * X[rr * 4 + rr];   // X[rr][rr] = 1/R[rr][rr], set earlier
    }
  }
}

}  // namespace tbkry
