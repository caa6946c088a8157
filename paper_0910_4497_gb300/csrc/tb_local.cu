// Exact gradient of the truncated local free energy at Krylov order
// r = r_min (the differentiable form of the method).
//
// Once r reaches the minimal-polynomial degree the block Krylov space of a
// target (Sec. 3, Eq. (Krylov)) is invariant and its projection is exact, so
// the target's spectral record is the dense eigen-decomposition of its cluster
// Hamiltonian H_c = Z diag(lam) Z^T (Sec. 2, locality).  Its grand potential
// Omega_i = 2 sum_a <i a|omega(H_c)|i a>, omega' = f, has the gradient
// (Daleckii-Krein)
//   dOmega_i/dH_c = 2 Z (Gamma o S^T S) Z^T,   S = Z[0:4, :],
//   Gamma_mk = (omega(lam_m) - omega(lam_k)) / (lam_m - lam_k),  Gamma_mm = f(lam_m),
// and every block of H_c depends on its bond vector, so the force terms of
// target i come from the 4x4 blocks of that matrix on the cluster's bonds.
// At fixed electron count d(sum_i A_i)/dR = d(sum_i Omega_i)/dR at fixed mu.
//
// One CTA per target (persistent over targets), everything in the CTA's slot
// of global workspace (the matrices are 4 n_c x 4 n_c, up to 512 x 512):
//   1. dense H_c from the bond blocks;
//   2. Householder reduction to tridiagonal form (row-oriented, one reflector
//      per step; each step's symmetric rank-2 update of the trailing block is
//      fused with the next step's matrix-vector product, one pass per step);
//   3. eigenvalues of the tridiagonal matrix by FP32 bisection on Sturm counts,
//      one thread per eigenvalue;
//   4. eigenvectors by inverse iteration with a pivoted tridiagonal LU (the
//      scheme of LAPACK's dlagtf/dlagts/dstein: three solves from a fixed start
//      vector, then Gram-Schmidt inside clusters of eigenvalues closer than
//      1e-3 ||T||), one thread per eigenvector, in the context precision;
//   5. FP64 Rayleigh quotients on the tridiagonal matrix;
//   6. back-transformation Z = Q Z_T: every warp keeps a few columns in
//      registers and applies the reflectors, staged 16 at a time in shared
//      memory;
// then, for the gradient:
//   7. M = Gamma o (S^T S) (Gamma in FP64, divided differences below 1e-3 kT by
//      the midpoint expansion f(c) + f''(c) d^2/24);
//   8. W = Z M (tiled shared-memory GEMM);
//   9. per directed bond (a -> b) inside the cluster, one warp: the block
//      G_ab = 2 W[a rows] Z[b rows]^T contracted with dH_ab/dd;
//  10. per cluster slot, the sum of its bonds' terms (fixed order) -> Floc;
// and a gather kernel adds, per atom, the terms of every target whose cluster
// holds it (clusters are symmetric: k in cluster(i) iff i in cluster(k)) plus
// the pair repulsion, in a fixed order.
#include "tb_internal.cuh"
#include "tb_model.cuh"

namespace {

constexpr int LT = 512;          // threads per CTA
constexpr int LW = LT / 32;      // warps per CTA
constexpr int RC = 16;           // reflectors staged per chunk (back-transformation)
constexpr int GT = 64;           // GEMM output tile (GT x GT)
constexpr int GK = 16;           // GEMM k chunk

template <typename TE> struct Cpw;                   // columns per warp, back-transformation
template <> struct Cpw<float> { static constexpr int v = 4; };
template <> struct Cpw<double> { static constexpr int v = 2; };

__device__ __forceinline__ double fermi_d(double x) {
  if (x > 50.0) return 0.0;
  if (x < -50.0) return 1.0;
  if (x > 0.0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

__device__ __forceinline__ double entropy_d(double f) {
  double t = 0.0;
  if (f > 0.0) t += f * log(f);
  if (f < 1.0) t += (1.0 - f) * log(1.0 - f);
  return t;
}

// omega(lam) = -kT ln(1 + e^{-x}), x = (lam - mu)/kT, without overflow
__device__ __forceinline__ double omega_d(double lam, double mu, double kT) {
  const double x = (lam - mu) / kT;
  if (x >= 0.0) return -kT * log1p(exp(-x));
  return (lam - mu) - kT * log1p(exp(x));
}

template <typename TE>
struct LocArgs {
  int n, ND, MH;
  const int *c_off, *c_idx, *h_off, *h_idx;
  const double *Hblk, *dHblk;
  double Es, Ep;
  TE *A, *Zw, *X;            // per slot: ND*ND, ND*ND, 5*ND*ND
  double* Cb;                // per slot: (ND/4)*MH*3
  double* lambda;            // n*ND
  double* S;                 // n*4*ND
  int* kdim;                 // n
  TE* Zstore;                // n*ND*ND or null
  const double* mu;
  double kT;
  double* Floc;              // n*(ND/4)*3
  int* st;
};

// shared-memory layout (bytes from the start of the dynamic block)
template <typename TE>
struct LocSmem {
  TE *v, *p, *dd, *ee, *tau, *sc, *vbuf, *Ssh, *ga, *gb;
  float *d32, *e2, *lam32;
  double *l64, *fd, *omd;
  int* cnt;
};

template <typename TE>
__host__ __device__ inline size_t loc_smem_bytes(int ND, LocSmem<TE>* out, unsigned char* base) {
  size_t off = 0;
  auto take = [&](size_t bytes) {
    unsigned char* p = base ? base + off : nullptr;
    off += (bytes + 15) & ~size_t(15);
    return p;
  };
  LocSmem<TE> s;
  s.v = reinterpret_cast<TE*>(take(sizeof(TE) * ND));
  s.p = reinterpret_cast<TE*>(take(sizeof(TE) * ND));
  s.dd = reinterpret_cast<TE*>(take(sizeof(TE) * ND));
  s.ee = reinterpret_cast<TE*>(take(sizeof(TE) * ND));
  s.tau = reinterpret_cast<TE*>(take(sizeof(TE) * ND));
  s.sc = reinterpret_cast<TE*>(take(sizeof(TE) * 64));
  s.vbuf = reinterpret_cast<TE*>(take(sizeof(TE) * RC * ND));
  s.Ssh = reinterpret_cast<TE*>(take(sizeof(TE) * 4 * ND));
  s.ga = reinterpret_cast<TE*>(take(sizeof(TE) * GT * (GK + 1)));
  s.gb = reinterpret_cast<TE*>(take(sizeof(TE) * GK * GT));
  s.d32 = reinterpret_cast<float*>(take(sizeof(float) * ND));
  s.e2 = reinterpret_cast<float*>(take(sizeof(float) * ND));
  s.lam32 = reinterpret_cast<float*>(take(sizeof(float) * ND));
  s.l64 = reinterpret_cast<double*>(take(sizeof(double) * ND));
  s.fd = reinterpret_cast<double*>(take(sizeof(double) * ND));
  s.omd = reinterpret_cast<double*>(take(sizeof(double) * ND));
  s.cnt = reinterpret_cast<int*>(take(sizeof(int) * 64));
  if (out) *out = s;
  return off;
}

// position of atom j in target i's cluster list (target first, then ascending), or -1
__device__ __forceinline__ int cluster_slot(const int* cl, int nc, int i, int j) {
  if (j == i) return 0;
  int lo = 1, hi = nc;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cl[mid] < j) lo = mid + 1; else hi = mid;
  }
  return (lo < nc && cl[lo] == j) ? lo : -1;
}

// position of atom j in the Hamiltonian list of atom a, or -1
__device__ __forceinline__ int hlist_pos(const int* h_off, const int* h_idx, int a, int j) {
  int lo = h_off[a], hi = h_off[a + 1];
  const int end = hi;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (h_idx[mid] < j) lo = mid + 1; else hi = mid;
  }
  return (lo < end && h_idx[lo] == j) ? lo : -1;
}

template <typename TE>
__device__ __forceinline__ TE warp_sum_t(TE v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// ---------------------------------------------------------------- 1. H_c

template <typename TE>
__device__ void build_hc(const LocArgs<TE>& a, int i, int nc, int nd, TE* A) {
  const int* cl = a.c_idx + a.c_off[i];
  for (int q = threadIdx.x; q < nd * nd; q += LT) A[q] = TE(0);
  __syncthreads();
  for (int x = threadIdx.x; x < nd; x += LT) A[(size_t)x * nd + x] = TE((x & 3) ? a.Ep : a.Es);
  for (int q = threadIdx.x; q < nc * a.MH; q += LT) {
    const int s = q / a.MH, k = q - s * a.MH;
    const int at = cl[s];
    const int p0 = a.h_off[at];
    if (k >= a.h_off[at + 1] - p0) continue;
    const int t = cluster_slot(cl, nc, i, a.h_idx[p0 + k]);
    if (t < 0) continue;
    const double* hb = a.Hblk + (size_t)(p0 + k) * 16;
#pragma unroll
    for (int al = 0; al < 4; ++al)
#pragma unroll
      for (int be = 0; be < 4; ++be) A[(size_t)(4 * s + al) * nd + 4 * t + be] = TE(hb[al * 4 + be]);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- 2. tridiagonal form

// Row-oriented Householder reduction of the symmetric A (nd x nd, full storage):
// reflector q maps row q's part right of the diagonal, A[q][q+1:], to
// (beta, 0, ..., 0) with H_q = I - tau_q v_q v_q^T (v_q[0] = 1), stored in
// A[q][q+2:] (v) and tau[q]; diagonal dd, off-diagonal ee.
//
// Step k (k = -1 .. nd-3) works on the trailing block A22 = A[k+1:, k+1:]
// (m = nd-k-1) and fuses reflector k's symmetric rank-2 update
//   A22 -= v w^T + w v^T,  p = tau A22 v,  w = p - (tau/2)(p.v) v,
// with the next step's product p' = tau' A33 v' (A33 = A22[1:, 1:]): warp 0
// first updates row k+1 and forms reflector k+1 from it; then every warp
// updates its rows of A33 and, while a row is still in registers, takes its
// dot product with v'.  The trailing block is read and written once per
// step; each lane keeps RB rows' columns in flight (RB x NI loads).  The
// column vectors v, w, v' sit in registers for FP32, in shared memory for
// FP64.  (Column 0 of A33's rows, below the new off-diagonal, is never read
// again and is left stale.)
template <typename TE>
__device__ void tridiagonalize(TE* A, int nd, const LocSmem<TE>& s) {
  constexpr int NI = 16;                       // columns per lane (nd <= 512)
  constexpr bool REG = sizeof(TE) == 4;        // column vectors in registers
  constexpr int RB = REG ? 2 : 1;              // rows per warp in flight
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  TE* const V[2] = {s.v, s.vbuf};              // reflector q in V[q & 1]
  TE* const P[2] = {s.p, s.vbuf + nd};         // its product tau_q A22 v_q in P[q & 1]
  for (int k = -1; k + 2 < nd; ++k) {
    const int m = nd - k - 1;
    TE* const base = A + (size_t)(k + 1) * (nd + 1);
    const bool has_next = m >= 3;              // reflector k+1 exists
    const TE t = k >= 0 ? s.sc[k & 1] : TE(0);
    const bool upd = t != TE(0);               // uniform
    const TE* vc = V[k & 1];
    const TE* pc = P[k & 1];
    TE* vn = V[(k + 1) & 1];
    TE* pn = P[(k + 1) & 1];
    TE c = TE(0);
    if (upd) {
      TE pv = TE(0);
      for (int j = lane; j < m; j += 32) pv += pc[j] * vc[j];
      c = TE(0.5) * t * warp_sum_t(pv);
    }
    // row k+1: reflector k's update, then reflector k+1
    if (warp == 0) {
      TE y[NI];
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int j = lane + 32 * i;
        y[i] = j < m ? base[j] : TE(0);
      }
      if (upd) {
        const TE v0 = vc[0], w0 = pc[0] - c * v0;
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          const int j = lane + 32 * i;
          if (j < m) {
            const TE vj = vc[j];
            y[i] -= v0 * (pc[j] - c * vj) + w0 * vj;
          }
        }
      }
      if (has_next) {
        TE sg = TE(0);
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          const int j = lane + 32 * i;
          if (j >= 2 && j < m) sg += y[i] * y[i];
        }
        sg = warp_sum_t(sg);
        const TE alpha = __shfl_sync(0xffffffffu, y[0], 1);
        TE beta = alpha, tn = TE(0), scale = TE(0);
        if (sg > TE(0)) {
          const TE nrm = sqrt(alpha * alpha + sg);
          beta = alpha <= TE(0) ? nrm : -nrm;
          tn = (beta - alpha) / beta;
          scale = TE(1) / (alpha - beta);
        }
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          const int j = lane + 32 * i;
          if (j >= 2 && j < m) {
            y[i] *= scale;
            vn[j - 1] = y[i];
          }
        }
        if (lane == 0) {
          vn[0] = TE(1);
          s.dd[k + 1] = y[0];
          s.ee[k + 1] = beta;
          s.tau[k + 1] = tn;
          s.sc[(k + 1) & 1] = tn;
        }
      }
#pragma unroll
      for (int i = 0; i < NI; ++i) {
        const int j = lane + 32 * i;
        if (j < m) base[j] = y[i];
      }
    }
    __syncthreads();
    const TE tn = has_next ? s.sc[(k + 1) & 1] : TE(0);
    const bool dot = tn != TE(0);              // uniform
    if (upd || dot) {
      // columns j = 1 + lane + 32 i of A22 (j < m): v_j, w_j, v'_{j-1}
      TE cv[REG ? NI : 1], cw[REG ? NI : 1], cn[REG ? NI : 1];
      if constexpr (REG) {
#pragma unroll
        for (int i = 0; i < NI; ++i) {
          const int j = 1 + lane + 32 * i;
          const bool in = j < m;
          cv[i] = in && upd ? vc[j] : TE(0);
          cw[i] = in && upd ? pc[j] - c * vc[j] : TE(0);
          cn[i] = in && dot ? vn[j - 1] : TE(0);
        }
      }
      for (int r0 = 1 + RB * warp; r0 < m; r0 += RB * LW) {
        TE x[RB][NI];
#pragma unroll
        for (int b = 0; b < RB; ++b) {
          const TE* row = base + (size_t)(r0 + b) * nd + 1;
#pragma unroll
          for (int i = 0; i < NI; ++i) {
            const int j = 1 + lane + 32 * i;
            x[b][i] = (r0 + b < m && j < m) ? row[j - 1] : TE(0);
          }
        }
        if (upd) {
#pragma unroll
          for (int b = 0; b < RB; ++b) {
            const int r = r0 + b < m ? r0 + b : 0;
            const TE vr = vc[r], wr = pc[r] - c * vr;
#pragma unroll
            for (int i = 0; i < NI; ++i) {
              if constexpr (REG) {
                x[b][i] -= vr * cw[i] + wr * cv[i];
              } else {
                const int j = 1 + lane + 32 * i;
                if (j < m) {
                  const TE vj = vc[j];
                  x[b][i] -= vr * (pc[j] - c * vj) + wr * vj;
                }
              }
            }
          }
#pragma unroll
          for (int b = 0; b < RB; ++b) {
            TE* row = base + (size_t)(r0 + b) * nd + 1;
#pragma unroll
            for (int i = 0; i < NI; ++i) {
              const int j = 1 + lane + 32 * i;
              if (r0 + b < m && j < m) row[j - 1] = x[b][i];
            }
          }
        }
        if (dot) {
          TE acc[RB];
#pragma unroll
          for (int b = 0; b < RB; ++b) {
            acc[b] = TE(0);
#pragma unroll
            for (int i = 0; i < NI; ++i) {
              if constexpr (REG) {
                acc[b] += x[b][i] * cn[i];
              } else {
                const int j = 1 + lane + 32 * i;
                if (j < m) acc[b] += x[b][i] * vn[j - 1];
              }
            }
          }
#pragma unroll
          for (int b = 0; b < RB; ++b) acc[b] = warp_sum_t(acc[b]);
          if (lane == 0) {
#pragma unroll
            for (int b = 0; b < RB; ++b)
              if (r0 + b < m) pn[r0 + b - 1] = tn * acc[b];
          }
        }
      }
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    if (nd >= 2) {
      s.dd[nd - 2] = A[(size_t)(nd - 2) * nd + nd - 2];
      s.ee[nd - 2] = A[(size_t)(nd - 2) * nd + nd - 1];
      s.tau[nd - 2] = TE(0);
    }
    s.dd[nd - 1] = A[(size_t)(nd - 1) * nd + nd - 1];
    s.ee[nd - 1] = TE(0);
    s.tau[nd - 1] = TE(0);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- 3-5. tridiagonal eigenpairs

__device__ __forceinline__ int sturm_count(const float* d, const float* e2, int n, float x,
                                           float pivmin) {
  float q = d[0] - x;
  if (fabsf(q) < pivmin) q = -pivmin;
  int cnt = q < 0.f;
  for (int i = 1; i < n; ++i) {
    q = d[i] - x - e2[i - 1] * __frcp_rn(q);
    if (fabsf(q) < pivmin) q = -pivmin;
    cnt += q < 0.f;
  }
  return cnt;
}

// start vector of inverse iteration (deterministic, all components nonzero)
__device__ __forceinline__ float start_component(int i, int e) {
  unsigned h = (unsigned)i * 2654435761u ^ ((unsigned)e * 40503u + 0x9e3779b9u);
  h ^= h >> 13;
  h *= 0x5bd1e995u;
  h ^= h >> 15;
  return 0.5f + (float)(h & 1023u) * (1.0f / 1023.0f);
}

// Eigenpairs of the tridiagonal (dd, ee) in the CTA: eigenvectors as the
// columns of Zw (nd x nd, [row][eigen]), FP64 eigenvalues in s.l64.
template <typename TE>
__device__ void tridiagonal_eigen(int nd, TE* Zw, TE* X, const LocSmem<TE>& s, int* st, int target) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t P = (size_t)nd * nd;
  TE* Xa = X;            // 1 / pivots of U
  TE* Xb = X + P;        // first super-diagonal of U
  TE* Xd = X + 2 * P;    // second super-diagonal of U (from interchanges)
  TE* Xc = X + 3 * P;    // multipliers of L
  TE* Xp = X + 4 * P;    // 1 where rows were interchanged
  // FP32 copies and Gershgorin bounds
  float gl = 1e30f, gu = -1e30f, e2max = 0.f;
  for (int x = tid; x < nd; x += LT) {
    const float dx = (float)s.dd[x];
    const float el = x > 0 ? fabsf((float)s.ee[x - 1]) : 0.f;
    const float er = x + 1 < nd ? fabsf((float)s.ee[x]) : 0.f;
    s.d32[x] = dx;
    s.e2[x] = er * er;
    e2max = fmaxf(e2max, er * er);
    gl = fminf(gl, dx - el - er);
    gu = fmaxf(gu, dx + el + er);
  }
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) {
    gl = fminf(gl, __shfl_xor_sync(0xffffffffu, gl, o));
    gu = fmaxf(gu, __shfl_xor_sync(0xffffffffu, gu, o));
    e2max = fmaxf(e2max, __shfl_xor_sync(0xffffffffu, e2max, o));
  }
  float* red = reinterpret_cast<float*>(s.cnt);
  if (lane == 0) {
    red[3 * warp] = gl;
    red[3 * warp + 1] = gu;
    red[3 * warp + 2] = e2max;
  }
  __syncthreads();
  gl = 1e30f;
  gu = -1e30f;
  e2max = 0.f;
  for (int w = 0; w < LW; ++w) {
    gl = fminf(gl, red[3 * w]);
    gu = fmaxf(gu, red[3 * w + 1]);
    e2max = fmaxf(e2max, red[3 * w + 2]);
  }
  const float tnorm = fmaxf(fmaxf(fabsf(gl), fabsf(gu)), 1e-30f);
  const float pivmin = 1e-30f * fmaxf(1.f, e2max);
  gl -= 2.4e-6f * tnorm + pivmin;
  gu += 2.4e-6f * tnorm + pivmin;
  // eigenvalues: bisection, one thread per eigenvalue
  for (int k = tid; k < nd; k += LT) {
    float lo = gl, hi = gu;
    for (int it = 0; it < 80; ++it) {
      if (hi - lo <= 1.2e-7f * fmaxf(fabsf(lo), fabsf(hi)) + pivmin) break;
      const float mid = 0.5f * (lo + hi);
      if (mid <= lo || mid >= hi) break;
      if (sturm_count(s.d32, s.e2, nd, mid, pivmin) > k) hi = mid; else lo = mid;
    }
    s.lam32[k] = 0.5f * (lo + hi);
  }
  __syncthreads();
  // eigenvectors: pivoted LU of T - sigma I, three solves.  The factors (five
  // nd x nd arrays, 3 MB per CTA in FP32) are stored and read with evict-first
  // hints so that they do not push the CTAs' matrix slots out of L2.
  const TE tiny = TE(tnorm) * TE(sizeof(TE) == 4 ? 1.2e-7 : 2.3e-16);
  for (int e = tid; e < nd; e += LT) {
    const TE sig = TE(s.lam32[e]);
    TE ak = s.dd[0] - sig;                 // current diagonal entry of row k
    TE bk = nd > 1 ? s.ee[0] : TE(0);      // current super-diagonal entry of row k
    for (int k = 0; k + 1 < nd; ++k) {
      const TE ck = s.ee[k];               // sub-diagonal entry (row k+1, column k)
      const TE ak1 = s.dd[k + 1] - sig;
      const TE bk1 = k + 2 < nd ? s.ee[k + 1] : TE(0);
      const size_t q = (size_t)k * nd + e;
      if (fabs(ak) >= fabs(ck)) {          // no interchange
        const TE piv = fabs(ak) < tiny ? (ak < TE(0) ? -tiny : tiny) : ak;
        const TE mult = ck / piv;
        __stcs(&Xa[q], TE(1) / piv);
        __stcs(&Xb[q], bk);
        __stcs(&Xd[q], TE(0));
        __stcs(&Xc[q], mult);
        __stcs(&Xp[q], TE(0));
        ak = ak1 - mult * bk;
        bk = bk1;
      } else {                             // rows k and k+1 interchanged
        const TE mult = ak / ck;
        __stcs(&Xa[q], TE(1) / ck);
        __stcs(&Xb[q], ak1);
        __stcs(&Xd[q], bk1);
        __stcs(&Xc[q], mult);
        __stcs(&Xp[q], TE(1));
        ak = bk - mult * ak1;
        bk = -mult * bk1;
      }
    }
    {
      const TE piv = fabs(ak) < tiny ? (ak < TE(0) ? -tiny : tiny) : ak;
      __stcs(&Xa[(size_t)(nd - 1) * nd + e], TE(1) / piv);
    }
    for (int x = 0; x < nd; ++x) Zw[(size_t)x * nd + e] = TE(start_component(x, e));
  }
  // every thread reads only its own eigenvector's factors: no barrier needed
  for (int it = 0; it < 3; ++it) {
    for (int e = tid; e < nd; e += LT) {
      // forward: apply the row interchanges and L^-1
      TE yk = Zw[e];
      for (int k = 0; k + 1 < nd; ++k) {
        const size_t q = (size_t)k * nd + e;
        const TE yk1 = Zw[q + nd];
        const TE mult = __ldcs(&Xc[q]);
        if (__ldcs(&Xp[q]) == TE(0)) {
          Zw[q] = yk;
          yk = yk1 - mult * yk;
        } else {
          Zw[q] = yk1;
          yk = yk - mult * yk1;
        }
      }
      Zw[(size_t)(nd - 1) * nd + e] = yk;
      // back substitution with U (diagonal given by reciprocals)
      TE y2 = TE(0), y1 = TE(0), nrm = TE(0);
      for (int k = nd - 1; k >= 0; --k) {
        const size_t q = (size_t)k * nd + e;
        TE y = Zw[q];
        if (k + 1 < nd) y -= __ldcs(&Xb[q]) * y1;
        if (k + 2 < nd) y -= __ldcs(&Xd[q]) * y2;
        y *= __ldcs(&Xa[q]);
        Zw[q] = y;
        y2 = y1;
        y1 = y;
        nrm += y * y;
      }
      const TE sc = TE(1) / sqrt(nrm);
      for (int x = 0; x < nd; ++x) Zw[(size_t)x * nd + e] *= sc;
    }
  }
  __syncthreads();
  // Gram-Schmidt inside clusters (one warp per cluster; members are consecutive)
  const float gtol = 1e-3f * tnorm;
  {
    int cl = 0;
    for (int e = 0; e < nd; ++e) {
      const bool start = (e == 0 || s.lam32[e] - s.lam32[e - 1] >= gtol);
      if (!start) continue;
      int end = e + 1;
      while (end < nd && s.lam32[end] - s.lam32[end - 1] < gtol) ++end;
      if (end - e > 1 && (cl++ % LW) == warp) {
        for (int b = e; b < end; ++b) {
          for (int a0 = e; a0 < b; ++a0) {
            TE dt = TE(0);
            for (int x = lane; x < nd; x += 32) dt += Zw[(size_t)x * nd + a0] * Zw[(size_t)x * nd + b];
            dt = warp_sum_t(dt);
            for (int x = lane; x < nd; x += 32) Zw[(size_t)x * nd + b] -= dt * Zw[(size_t)x * nd + a0];
            __syncwarp();
          }
          TE nn = TE(0);
          for (int x = lane; x < nd; x += 32) nn += Zw[(size_t)x * nd + b] * Zw[(size_t)x * nd + b];
          nn = warp_sum_t(nn);
          const TE sc = TE(1) / sqrt(nn);
          for (int x = lane; x < nd; x += 32) Zw[(size_t)x * nd + b] *= sc;
          __syncwarp();
        }
      }
    }
  }
  __syncthreads();
  // FP64 Rayleigh quotients on the tridiagonal matrix
  for (int e = tid; e < nd; e += LT) {
    double num = 0.0, den = 0.0, zp = 0.0;
    for (int x = 0; x < nd; ++x) {
      const double z = (double)Zw[(size_t)x * nd + e];
      num += (double)s.dd[x] * z * z;
      if (x > 0) num += 2.0 * (double)s.ee[x - 1] * zp * z;
      den += z * z;
      zp = z;
    }
    const double l = num / den;
    s.l64[e] = l;
    if (!isfinite(l)) tbk::set_status(st, TB_ERR_NONFINITE, target);
  }
  __syncthreads();
}

// ---------------------------------------------------------------- 6. back-transformation

// Zw <- Q Zw with Q = H_0 H_1 ... H_{nd-3}; reflector k acts on rows k+1..nd-1.
template <typename TE>
__device__ void back_transform(const TE* A, int nd, TE* Zw, const LocSmem<TE>& s) {
  constexpr int CPW = Cpw<TE>::v;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int nref = nd - 2;                // reflectors 0..nd-3
  const int rows_pl = (nd + 31) >> 5;     // rows per lane, <= 16
  for (int j0 = 0; j0 < nd; j0 += LW * CPW) {
    TE z[CPW][16];
    const int jw = j0 + warp * CPW;
#pragma unroll
    for (int c = 0; c < CPW; ++c)
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int x = lane + 32 * t;
        z[c][t] = (t < rows_pl && x < nd && jw + c < nd) ? Zw[(size_t)x * nd + jw + c] : TE(0);
      }
    for (int k1 = nref - 1; k1 >= 0; k1 -= RC) {
      const int k0 = k1 - RC + 1 < 0 ? 0 : k1 - RC + 1;
      const int nr = k1 - k0 + 1;
      __syncthreads();
      for (int q = tid; q < nr * nd; q += LT) {
        const int r = q / nd, x = q - r * nd;
        const int k = k1 - r;
        TE v = TE(0);
        if (x == k + 1) v = TE(1);
        else if (x > k + 1) v = A[(size_t)k * nd + x];
        s.vbuf[r * nd + x] = v;
      }
      __syncthreads();
      for (int r = 0; r < nr; ++r) {
        const int k = k1 - r;
        const TE t = s.tau[k];
        if (t == TE(0)) continue;
        const TE* vr = s.vbuf + r * nd;
        TE y[CPW];
#pragma unroll
        for (int c = 0; c < CPW; ++c) y[c] = TE(0);
#pragma unroll
        for (int tt = 0; tt < 16; ++tt) {
          const int x = lane + 32 * tt;
          if (tt < rows_pl && x < nd) {
            const TE vx = vr[x];
#pragma unroll
            for (int c = 0; c < CPW; ++c) y[c] += vx * z[c][tt];
          }
        }
#pragma unroll
        for (int c = 0; c < CPW; ++c) y[c] = t * warp_sum_t(y[c]);
#pragma unroll
        for (int tt = 0; tt < 16; ++tt) {
          const int x = lane + 32 * tt;
          if (tt < rows_pl && x < nd) {
            const TE vx = vr[x];
#pragma unroll
            for (int c = 0; c < CPW; ++c) z[c][tt] -= vx * y[c];
          }
        }
      }
    }
#pragma unroll
    for (int c = 0; c < CPW; ++c)
#pragma unroll
      for (int t = 0; t < 16; ++t) {
        const int x = lane + 32 * t;
        if (t < rows_pl && x < nd && jw + c < nd) Zw[(size_t)x * nd + jw + c] = z[c][t];
      }
  }
  __syncthreads();
}

// Dense eigen-decomposition of target i's H_c: Z in Zw (nd x nd, [row][m]),
// FP64 eigenvalues (ascending) in s.l64.
template <typename TE>
__device__ void eigh_target(const LocArgs<TE>& a, int i, int nc, int nd, TE* A, TE* Zw, TE* X,
                            const LocSmem<TE>& s) {
  build_hc(a, i, nc, nd, A);
  tridiagonalize(A, nd, s);
  tridiagonal_eigen(nd, Zw, X, s, a.st, i);
  back_transform(A, nd, Zw, s);
}

// ---------------------------------------------------------------- forward kernel

template <typename TE>
__global__ void __launch_bounds__(LT, 1) local_spectrum_kernel(const LocArgs<TE> a) {
  extern __shared__ __align__(16) unsigned char loc_smem[];
  LocSmem<TE> s;
  loc_smem_bytes<TE>(a.ND, &s, loc_smem);
  const size_t slot = blockIdx.x;
  const size_t N2 = (size_t)a.ND * a.ND;
  TE* A = a.A + slot * N2;
  TE* Zw = a.Zw + slot * N2;
  TE* X = a.X + slot * 5 * N2;
  for (int i = blockIdx.x; i < a.n; i += gridDim.x) {
    const int nc = a.c_off[i + 1] - a.c_off[i];
    const int nd = 4 * nc;
    if (nc < 1 || nd > a.ND) {
      if (threadIdx.x == 0) tbk::set_status(a.st, TB_ERR_CAPACITY, nd);
      continue;
    }
    eigh_target(a, i, nc, nd, A, Zw, X, s);
    double* lo = a.lambda + (size_t)i * a.ND;
    double* So = a.S + (size_t)i * 4 * a.ND;
    for (int k = threadIdx.x; k < a.ND; k += LT) {
      lo[k] = k < nd ? s.l64[k] : 0.0;
#pragma unroll
      for (int al = 0; al < 4; ++al) So[al * a.ND + k] = k < nd ? (double)Zw[(size_t)al * nd + k] : 0.0;
    }
    if (threadIdx.x == 0) a.kdim[i] = nd;
    if (a.Zstore) {
      TE* zo = a.Zstore + (size_t)i * N2;
      for (int q = threadIdx.x; q < nd * nd; q += LT) zo[q] = Zw[q];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- gradient kernel

// W = Z M for nd x nd row-major matrices (tiled through shared memory)
template <typename TE>
__device__ void gemm_nn(const TE* Z, const TE* M, TE* W, int nd, const LocSmem<TE>& s) {
  const int tid = threadIdx.x;
  const int tr = tid >> 4, tc = tid & 15;          // 32 x 16 thread grid: 2 rows x 4 cols each
  for (int r0 = 0; r0 < nd; r0 += GT)
    for (int c0 = 0; c0 < nd; c0 += GT) {
      TE acc[2][4];
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) acc[u][v] = TE(0);
      for (int k0 = 0; k0 < nd; k0 += GK) {
        __syncthreads();
        for (int q = tid; q < GT * GK; q += LT) {
          const int r = q / GK, kk = q - r * GK;
          const int gr = r0 + r, gk = k0 + kk;
          s.ga[r * (GK + 1) + kk] = (gr < nd && gk < nd) ? Z[(size_t)gr * nd + gk] : TE(0);
          const int kb = q / GT, cc = q - kb * GT;
          const int gkb = k0 + kb, gc = c0 + cc;
          s.gb[kb * GT + cc] = (gkb < nd && gc < nd) ? M[(size_t)gkb * nd + gc] : TE(0);
        }
        __syncthreads();
#pragma unroll
        for (int kk = 0; kk < GK; ++kk) {
          const TE a0 = s.ga[(2 * tr) * (GK + 1) + kk], a1 = s.ga[(2 * tr + 1) * (GK + 1) + kk];
#pragma unroll
          for (int v = 0; v < 4; ++v) {
            const TE b = s.gb[kk * GT + tc + 16 * v];
            acc[0][v] += a0 * b;
            acc[1][v] += a1 * b;
          }
        }
      }
#pragma unroll
      for (int u = 0; u < 2; ++u)
#pragma unroll
        for (int v = 0; v < 4; ++v) {
          const int gr = r0 + 2 * tr + u, gc = c0 + tc + 16 * v;
          if (gr < nd && gc < nd) W[(size_t)gr * nd + gc] = acc[u][v];
        }
    }
  __syncthreads();
}

template <typename TE>
__global__ void __launch_bounds__(LT, 1) local_gradient_kernel(const LocArgs<TE> a) {
  extern __shared__ __align__(16) unsigned char loc_smem[];
  LocSmem<TE> s;
  loc_smem_bytes<TE>(a.ND, &s, loc_smem);
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const size_t slot = blockIdx.x;
  const size_t N2 = (size_t)a.ND * a.ND;
  TE* A = a.A + slot * N2;
  TE* Zw = a.Zw + slot * N2;
  TE* X = a.X + slot * 5 * N2;
  double* Cb = a.Cb + slot * (size_t)(a.ND / 4) * a.MH * 3;
  const double mu = *a.mu, kT = a.kT;
  for (int i = blockIdx.x; i < a.n; i += gridDim.x) {
    const int nc = a.c_off[i + 1] - a.c_off[i];
    const int nd = 4 * nc;
    const int* cl = a.c_idx + a.c_off[i];
    if (nc < 1 || nd > a.ND) {
      if (tid == 0) tbk::set_status(a.st, TB_ERR_CAPACITY, nd);
      continue;
    }
    const TE* Z = Zw;
    if (a.Zstore) Z = a.Zstore + (size_t)i * N2;
    else eigh_target(a, i, nc, nd, A, Zw, X, s);
    // per eigenpair: lam, f, omega (FP64) and the seed rows S
    const double* li = a.lambda + (size_t)i * a.ND;
    for (int k = tid; k < nd; k += LT) {
      const double l = li[k];
      s.l64[k] = l;
      s.fd[k] = fermi_d((l - mu) / kT);
      s.omd[k] = omega_d(l, mu, kT);
#pragma unroll
      for (int al = 0; al < 4; ++al) s.Ssh[al * nd + k] = Z[(size_t)al * nd + k];
    }
    __syncthreads();
    // M = Gamma o (S^T S) into X
    TE* M = X;
    const double ikT = 1.0 / kT;
    for (int q = tid; q < nd * nd; q += LT) {
      const int m = q / nd, k = q - m * nd;
      const double dl = s.l64[m] - s.l64[k];
      double g;
      if (fabs(dl) <= 1e-3 * kT) {
        const double fc = fermi_d((0.5 * (s.l64[m] + s.l64[k]) - mu) * ikT);
        g = fc + fc * (1.0 - fc) * (1.0 - 2.0 * fc) * dl * dl * ikT * ikT * (1.0 / 24.0);
      } else {
        g = (s.omd[m] - s.omd[k]) / dl;
      }
      double ss = 0.0;
#pragma unroll
      for (int al = 0; al < 4; ++al) ss += (double)s.Ssh[al * nd + m] * (double)s.Ssh[al * nd + k];
      M[q] = TE(g * ss);
    }
    __syncthreads();
    // W = Z M into A
    gemm_nn(Z, M, A, nd, s);
    // per directed bond inside the cluster: c = sum_ab G_ab dH_ab/dd, G_ab = 2 W_a Z_b^T
    for (int q = warp; q < nc * a.MH; q += LW) {
      const int sl = q / a.MH, kq = q - sl * a.MH;
      const int at = cl[sl];
      const int p0 = a.h_off[at];
      double* cq = Cb + (size_t)q * 3;
      int t = -1;
      if (kq < a.h_off[at + 1] - p0) t = cluster_slot(cl, nc, i, a.h_idx[p0 + kq]);
      if (t < 0) {
        if (lane < 3) cq[lane] = 0.0;
        continue;
      }
      TE acc[16];
#pragma unroll
      for (int v = 0; v < 16; ++v) acc[v] = TE(0);
      const TE* Wr = A + (size_t)(4 * sl) * nd;
      const TE* Zr = Z + (size_t)(4 * t) * nd;
      for (int m = lane; m < nd; m += 32) {
        TE wv[4], zv[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          wv[u] = Wr[(size_t)u * nd + m];
          zv[u] = Zr[(size_t)u * nd + m];
        }
#pragma unroll
        for (int al = 0; al < 4; ++al)
#pragma unroll
          for (int be = 0; be < 4; ++be) acc[al * 4 + be] += wv[al] * zv[be];
      }
      double accd[16];
#pragma unroll
      for (int v = 0; v < 16; ++v) accd[v] = (double)acc[v];
      const double g = tbk::warp_reduce16(accd, lane);   // lanes 2v hold G/2 entry v
      const double* dH = a.dHblk + (size_t)(p0 + kq) * 48;
      double c3[3] = {0.0, 0.0, 0.0};
      if ((lane & 1) == 0) {
        const int v = lane >> 1;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) c3[kk] = 2.0 * g * dH[kk * 16 + v];
      }
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) c3[kk] = tbk::warp_sum(c3[kk]);
      if (lane < 3) cq[lane] = c3[lane];
    }
    __syncthreads();
    // per slot: -dOmega_i/dR_slot = sum over its bonds (s -> t) of c - sum over (t -> s) of c
    double* Fo = a.Floc + (size_t)i * (a.ND / 4) * 3;
    for (int sl = tid; sl < nc; sl += LT) {
      const int at = cl[sl];
      const int p0 = a.h_off[at], deg = a.h_off[at + 1] - p0;
      double f[3] = {0.0, 0.0, 0.0};
      for (int kq = 0; kq < deg; ++kq) {
        const int j = a.h_idx[p0 + kq];
        const int t = cluster_slot(cl, nc, i, j);
        if (t < 0) continue;
        const int pr = hlist_pos(a.h_off, a.h_idx, j, at);
        const double* c1 = Cb + (size_t)(sl * a.MH + kq) * 3;
#pragma unroll
        for (int kk = 0; kk < 3; ++kk) f[kk] += c1[kk];
        if (pr >= 0) {
          const double* c2 = Cb + (size_t)(t * a.MH + (pr - a.h_off[j])) * 3;
#pragma unroll
          for (int kk = 0; kk < 3; ++kk) f[kk] -= c2[kk];
        } else {
          tbk::set_status(a.st, TB_ERR_INVALID_ARG, at);
        }
      }
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) Fo[(size_t)sl * 3 + kk] = f[kk];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------- energies, gather

struct LocEnergyArgs {
  int n, ND;
  const double *lambda, *S, *mu, *pos;
  double kT, L;
  const int *h_off, *h_idx;
  tb_gsp rep;
  double* per_target;
};

// per target: E_band, -TS, N_e of its dense record and half its bonds' repulsion
__global__ void __launch_bounds__(128) local_energy_kernel(const LocEnergyArgs a) {
  __shared__ double red[4 * 4];
  __shared__ double tot[4];
  const int i = blockIdx.x;
  const double mu = *a.mu;
  const double* lam = a.lambda + (size_t)i * a.ND;
  const double* Si = a.S + (size_t)i * 4 * a.ND;
  double v[4] = {0.0, 0.0, 0.0, 0.0};
  for (int k = threadIdx.x; k < a.ND; k += 128) {
    const double w = Si[k] * Si[k] + Si[a.ND + k] * Si[a.ND + k] +
                     Si[2 * a.ND + k] * Si[2 * a.ND + k] + Si[3 * a.ND + k] * Si[3 * a.ND + k];
    if (w == 0.0) continue;
    const double f = fermi_d((lam[k] - mu) / a.kT);
    v[0] += w * f * lam[k];
    v[1] += w * entropy_d(f);
    v[2] += w * f;
  }
  const int deg = a.h_off[i + 1] - a.h_off[i];
  if (threadIdx.x < deg) {
    const int j = a.h_idx[a.h_off[i] + threadIdx.x];
    const double hL = 0.5 * a.L;
    double d2 = 0.0;
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const double x = a.pos[3 * j + kk] - a.pos[3 * i + kk];
      const double dx = x > hL ? x - a.L : (x < -hL ? x + a.L : x);
      d2 += dx * dx;
    }
    double phi, dphi;
    tb_gsp_eval(a.rep, sqrt(d2), phi, dphi);
    v[3] = 0.5 * phi;
  }
  tbk::block_sum<double, 4>(v, red, tot);
  if (threadIdx.x == 0) {
    a.per_target[5 * i + 0] = 2.0 * tot[0];
    a.per_target[5 * i + 1] = 2.0 * a.kT * tot[1];
    a.per_target[5 * i + 2] = 2.0 * tot[2];
    a.per_target[5 * i + 3] = tot[3];
    a.per_target[5 * i + 4] = 0.0;
  }
}

struct GatherArgs {
  int n, ND;
  const int *c_off, *c_idx, *h_off, *h_idx;
  const double *Floc, *pos;
  double L;
  tb_gsp rep;
  double* F;
  int* st;
};

__global__ void __launch_bounds__(128) local_gather_kernel(const GatherArgs a) {
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  if (k >= a.n) return;
  double f[3] = {0.0, 0.0, 0.0};
  for (int q = a.c_off[k]; q < a.c_off[k + 1]; ++q) {
    const int i = a.c_idx[q];
    const int* cl = a.c_idx + a.c_off[i];
    const int sl = cluster_slot(cl, a.c_off[i + 1] - a.c_off[i], i, k);
    if (sl < 0) {
      tbk::set_status(a.st, TB_ERR_INVALID_ARG, k);
      continue;
    }
    const double* fo = a.Floc + ((size_t)i * (a.ND / 4) + sl) * 3;
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) f[kk] += fo[kk];
  }
  const double hL = 0.5 * a.L;
  for (int p = a.h_off[k]; p < a.h_off[k + 1]; ++p) {
    const int j = a.h_idx[p];
    double d[3];
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) {
      const double x = a.pos[3 * j + kk] - a.pos[3 * k + kk];
      d[kk] = x > hL ? x - a.L : (x < -hL ? x + a.L : x);
    }
    const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    double phi, dphi;
    tb_gsp_eval(a.rep, r, phi, dphi);
#pragma unroll
    for (int kk = 0; kk < 3; ++kk) f[kk] += dphi / r * d[kk];
  }
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) a.F[3 * k + kk] = f[kk];
  if (!(isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]))) tbk::set_status(a.st, TB_ERR_NONFINITE, k);
}

template <typename TE>
LocArgs<TE> loc_args(tb_ctx* c, int n, const int* c_off, const int* c_idx, const int* h_off,
                     const int* h_idx, const double* Hblk, const double* dHblk, double* lambda,
                     double* S, int* kdim, void* Zstore, const double* mu) {
  LocArgs<TE> a;
  a.n = n;
  a.ND = c->loc_ND;
  a.MH = c->p.max_hnbr;
  a.c_off = c_off;
  a.c_idx = c_idx;
  a.h_off = h_off;
  a.h_idx = h_idx;
  a.Hblk = Hblk;
  a.dHblk = dHblk;
  a.Es = c->p.Es;
  a.Ep = c->p.Ep;
  a.A = static_cast<TE*>(c->loc_A);
  a.Zw = static_cast<TE*>(c->loc_Z);
  a.X = static_cast<TE*>(c->loc_X);
  a.Cb = c->loc_Cb;
  a.lambda = lambda;
  a.S = S;
  a.kdim = kdim;
  a.Zstore = static_cast<TE*>(Zstore);
  a.mu = mu;
  a.kT = c->p.kT;
  a.Floc = c->loc_Floc;
  a.st = c->d_status;
  return a;
}

template <typename TE>
tb_status configure_local_t(tb_ctx* c) {
  const size_t smem = loc_smem_bytes<TE>(c->loc_ND, nullptr, nullptr);
  int max_smem = 0;
  TB_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, c->device));
  if (smem > (size_t)max_smem) return TB_ERR_CAPACITY;
  TB_CUDA_TRY(cudaFuncSetAttribute(local_spectrum_kernel<TE>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  TB_CUDA_TRY(cudaFuncSetAttribute(local_gradient_kernel<TE>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  c->loc_smem = smem;
  c->loc_grid = c->num_sms;
  c->loc_esize = sizeof(TE);
  return TB_OK;
}

}  // namespace

size_t local_workspace_bytes(tb_ctx* c, int n) {
  const size_t ND = c->loc_ND, G = c->loc_grid, es = c->loc_esize;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  return al(G * ND * ND * es) * 2 + al(G * 5 * ND * ND * es) +
         al(G * (ND / 4) * c->p.max_hnbr * 3 * sizeof(double)) +
         al((size_t)n * (ND / 4) * 3 * sizeof(double));
}

void local_carve(tb_ctx* c, int n, unsigned char* base) {
  const size_t ND = c->loc_ND, G = c->loc_grid, es = c->loc_esize;
  auto al = [](size_t x) { return (x + 255) & ~size_t(255); };
  size_t off = 0;
  c->loc_A = base + off;
  off += al(G * ND * ND * es);
  c->loc_Z = base + off;
  off += al(G * ND * ND * es);
  c->loc_X = base + off;
  off += al(G * 5 * ND * ND * es);
  c->loc_Cb = reinterpret_cast<double*>(base + off);
  off += al(G * (ND / 4) * c->p.max_hnbr * 3 * sizeof(double));
  c->loc_Floc = reinterpret_cast<double*>(base + off);
  (void)n;
}

tb_status local_configure(tb_ctx* c) {
  c->loc_ND = 4 * c->p.max_cluster;
  if (c->loc_ND > TB_LOCAL_MAX_DIM) return TB_ERR_CAPACITY;
  return c->p.prec == TB_PREC_FP64 ? configure_local_t<double>(c) : configure_local_t<float>(c);
}

tb_status launch_local_forward(tb_ctx* c, int n, const double* pos, double L, const int* c_off,
                               const int* c_idx, const int* h_off, const int* h_idx,
                               const double* Hblk, double* lambda, double* S, int* kdim,
                               void* Zstore, double* mu, double* energies, cudaStream_t s) {
  const int grid = n < c->loc_grid ? n : c->loc_grid;
  if (c->p.prec == TB_PREC_FP64) {
    auto a = loc_args<double>(c, n, c_off, c_idx, h_off, h_idx, Hblk, nullptr, lambda, S, kdim,
                              Zstore, mu);
    local_spectrum_kernel<double><<<grid, LT, c->loc_smem, s>>>(a);
  } else {
    auto a = loc_args<float>(c, n, c_off, c_idx, h_off, h_idx, Hblk, nullptr, lambda, S, kdim,
                             Zstore, mu);
    local_spectrum_kernel<float><<<grid, LT, c->loc_smem, s>>>(a);
  }
  TB_CUDA_TRY(cudaGetLastError());
  tb_status st = launch_mu_nt(c, n, c->loc_ND, lambda, S, 4.0 * n, nullptr, mu, nullptr, s);
  if (st != TB_OK) return st;
  LocEnergyArgs e{n, c->loc_ND, lambda, S, mu, pos, c->p.kT, L, h_off, h_idx,
                  tb_repulsion_gsp(c->p), c->per_target};
  local_energy_kernel<<<n, 128, 0, s>>>(e);
  TB_CUDA_TRY(cudaGetLastError());
  return launch_energy_reduce(n, c->per_target, mu, energies, s);
}

tb_status launch_local_gradient(tb_ctx* c, int n, const double* pos, double L, const int* c_off,
                                const int* c_idx, const int* h_off, const int* h_idx,
                                const double* Hblk, const double* dHblk, const double* lambda,
                                const double* S, const void* Zstore, const double* mu, double* F,
                                cudaStream_t s) {
  const int grid = n < c->loc_grid ? n : c->loc_grid;
  double* lam = const_cast<double*>(lambda);
  double* Sm = const_cast<double*>(S);
  void* Zs = const_cast<void*>(Zstore);
  if (c->p.prec == TB_PREC_FP64) {
    auto a = loc_args<double>(c, n, c_off, c_idx, h_off, h_idx, Hblk, dHblk, lam, Sm, nullptr,
                              Zs, mu);
    local_gradient_kernel<double><<<grid, LT, c->loc_smem, s>>>(a);
  } else {
    auto a = loc_args<float>(c, n, c_off, c_idx, h_off, h_idx, Hblk, dHblk, lam, Sm, nullptr,
                             Zs, mu);
    local_gradient_kernel<float><<<grid, LT, c->loc_smem, s>>>(a);
  }
  TB_CUDA_TRY(cudaGetLastError());
  GatherArgs g{n, c->loc_ND, c_off, c_idx, h_off, h_idx, c->loc_Floc, pos, L,
               tb_repulsion_gsp(c->p), F, c->d_status};
  local_gather_kernel<<<(n + 127) / 128, 128, 0, s>>>(g);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}
