// The m-target form of the block recursion (Sec. 3, Eq. (lanczos_blas3))
// and the spatial grouping of the targets it runs on.
//
// Grouping.  The atoms are sorted by (Morton code of their grid cell, index)
// and cut into consecutive groups of m.  The grid has g^3 cells, g the largest
// integer with m g^3 <= n (about m atoms per cell); an atom's cell is
// floor((x / L) * g) per component, clamped to [0, g-1]; bit b of the cell
// coordinates x, y, z goes to bits 3b, 3b+1, 3b+2 of the code.  The sort is a
// rank count (each atom counts the keys below its own), split over CTAs along
// the other atoms, then a scatter: integer work, identical on every run.
//
// Grouped block Lanczos.  One CTA per group of up to MC targets.  The group's
// shared matrix is the Hamiltonian of the union of its targets' clusters: the
// CTA concatenates the member clusters, sorts them (bitonic, in shared
// memory), drops repeats, and builds one local sparsity map of H_u.  Each
// target t keeps its own recursion (A_k, B_k block diagonal over the targets):
//   W_t = H_u V_{t,k} - V_{t,k-1} B_{t,k-1}^T          one sweep for all targets
//   classical Gram-Schmidt of W_t against V_{t,1..k}  per target
//   W_t = V_{t,k+1} B_{t,k}                          Cholesky QR per target,
//                                                    MGS with deflation when a
//                                                    pivot refuses
// The sweep reads each 4x4 block of H_u once for the 4*MC columns of all the
// targets (the Level-3 shape of Eq. (lanczos_blas3)).  A target whose block
// deflates to nothing drops out; the others continue.  Outputs per target are
// the same as the per-target kernel's: T, the rows of V for the target and its
// Hamiltonian neighbours (Y), the active-column mask.  The projected
// eigensolve that follows is the per-target one.
//
// Layout: the basis of target t lives in a per-CTA slot of global memory
// (L2-resident), block k of target t at V + (t r + k) * Dmax * 4, row-major
// [row][4]; W (and, when it fits, a staged copy of every V_k) in shared memory.
#include <climits>

#include "tb_internal.cuh"
#include "tb_krylov_common.cuh"

namespace {

using namespace tbkry;

constexpr int GMAX = 4;            // targets per group, at most
constexpr int UBUF_MAX = 4096;     // concatenated member lists, at most

__host__ __device__ __forceinline__ size_t al32(size_t x) { return (x + 31) & ~size_t(31); }

// ------------------------------------------------------------------ grouping

__device__ __forceinline__ unsigned morton3(unsigned cx, unsigned cy, unsigned cz) {
  unsigned code = 0;
#pragma unroll
  for (int b = 0; b < 10; ++b) {
    code |= ((cx >> b) & 1u) << (3 * b);
    code |= ((cy >> b) & 1u) << (3 * b + 1);
    code |= ((cz >> b) & 1u) << (3 * b + 2);
  }
  return code;
}

__device__ __forceinline__ unsigned long long group_key(const double* pos, int i, double L,
                                                        int g) {
  unsigned c[3];
#pragma unroll
  for (int d = 0; d < 3; ++d) {
    const double t = __dmul_rn(__ddiv_rn(pos[3 * i + d], L), (double)g);
    int ci = (int)floor(t);
    ci = ci < 0 ? 0 : (ci > g - 1 ? g - 1 : ci);
    c[d] = (unsigned)ci;
  }
  return ((unsigned long long)morton3(c[0], c[1], c[2]) << 32) | (unsigned)i;
}

// cnt[i] += number of atoms j in this CTA's slice with key_j < key_i
__global__ void __launch_bounds__(256) group_count_kernel(int n, const double* __restrict__ pos,
                                                          double L, int g, int per,
                                                          int* __restrict__ cnt) {
  __shared__ unsigned long long tile[256];
  const int i = blockIdx.x * 256 + threadIdx.x;
  const unsigned long long ki = i < n ? group_key(pos, i, L, g) : ~0ull;
  const int j0 = blockIdx.y * per;
  const int j1 = min(n, j0 + per);
  int c = 0;
  for (int base = j0; base < j1; base += 256) {
    const int j = base + threadIdx.x;
    tile[threadIdx.x] = j < j1 ? group_key(pos, j, L, g) : ~0ull;
    __syncthreads();
    const int cnt_t = min(256, j1 - base);
    for (int q = 0; q < cnt_t; ++q) c += tile[q] < ki;
    __syncthreads();
  }
  if (i < n && c) atomicAdd(cnt + i, c);
}

__global__ void group_scatter_kernel(int n, int m, const int* __restrict__ cnt,
                                     int* __restrict__ g_off, int* __restrict__ g_idx) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) g_idx[cnt[i]] = i;
  const int G = (n + m - 1) / m;
  if (i <= G) g_off[i] = min(i * m, n);
}

// ------------------------------------------------------------ grouped Lanczos

template <typename TV>
struct KryGArgs {
  int n, n_groups, r, max_cluster, max_union, max_hnbr, reorth_passes, reorth_every, ubuf;
  double Es, Ep, defl_tol;
  const int* g_off;
  const int* g_idx;
  const int* c_off;
  const int* c_idx;
  const int* h_off;
  const int* h_idx;
  const TV* H;                        // FP64: the bond blocks
  const float4* Hsk;                  // FP32: Slater-Koster records (s, l)
  float Vss, Vsp, Cpp, Vppp;          // Cpp = Vpps - Vppp
  double* T;                          // compact block-tridiagonal T
  TV* Y;
  unsigned long long* colmask;
  TV* Vg;
  int2* lent;
  int lent_smem;
  int* st;
};

// Row al of the 4x4 block of bond p: read from the FP64 table, or rebuilt
// from the FP32 Slater-Koster record (s, l) with the table of Eq. (1):
// row s = s (Vss, Vsp l), row p_g = s (-Vsp l_g, (Vpps - Vppp) l_g l + Vppp e_g).
template <typename TV>
__device__ __forceinline__ vec4<TV> hrow(const KryGArgs<TV>& a, int p, int al) {
  if constexpr (sizeof(TV) == 8) {
    return ldg4(a.H + (size_t)p * 16 + al * 4);
  } else {
    const float4 h = __ldg(a.Hsk + p);
    vec4<TV> o;
    if (al == 0) {
      const float sv = h.x * a.Vsp;
      o.v[0] = h.x * a.Vss; o.v[1] = sv * h.y; o.v[2] = sv * h.z; o.v[3] = sv * h.w;
    } else {
      const float lg = al == 1 ? h.y : (al == 2 ? h.z : h.w);
      const float t = h.x * a.Cpp * lg, d = h.x * a.Vppp;
      o.v[0] = -h.x * a.Vsp * lg;
      o.v[1] = fmaf(t, h.y, al == 1 ? d : 0.f);
      o.v[2] = fmaf(t, h.z, al == 2 ? d : 0.f);
      o.v[3] = fmaf(t, h.w, al == 3 ? d : 0.f);
    }
    return o;
  }
}

// integer scratch in shared memory
constexpr int GI_WT = 0;          // warp totals of the block scans (<= 16 warps)
constexpr int GI_MASK = 16;       // per target: basis column mask, two words
constexpr int GI_ACT = GI_MASK + 2 * GMAX;   // per target: active columns of the newest block
constexpr int GI_OK = GI_ACT + GMAX;         // per target: Cholesky-QR verdict
constexpr int GI_CS = GI_OK + GMAX;          // per target: 0, or the refused Cholesky pass
constexpr int GI_SLOT = GI_CS + GMAX;        // per target: slot in the union list
constexpr int GI_NB = GI_SLOT + GMAX;        // per target: basis blocks kept
constexpr int GI_LT = GI_NB + GMAX;          // live targets, in order
constexpr int GI_LIVE = GI_LT + GMAX;
constexpr int GI_NL = GI_LIVE + 1;
constexpr int GI_NU = GI_NL + 1;
constexpr int GI_SIZE = GI_NU + 1;

template <typename TV, int MC, int KT, bool VKS>
__host__ __device__ inline size_t kryg_smem_bytes(int r, int max_union, int max_hnbr, bool lsmem,
                                                  int ubuf) {
  constexpr int KW = KT / 32;
  constexpr int NCH = (10 * MC + 15) / 16;
  const size_t BS = 16 * (size_t)max_union;
  const size_t npi = (size_t)(MC * r > KW ? MC * r : KW);
  size_t b = 0;
  b += al32(sizeof(int) * ubuf);                         // concatenated lists / sort
  b += al32(sizeof(int) * max_union);                    // union list
  b += al32(sizeof(int) * (max_union + 1));              // rowptr
  b += al32(sizeof(TV) * MC * BS);                       // W
  if (VKS) b += al32(sizeof(TV) * MC * BS);              // staged V_k
  if (lsmem) b += al32(sizeof(int2) * (size_t)max_union * max_hnbr);
  b += al32(sizeof(TV) * 16 * npi);                      // projection partials
  b += al32(sizeof(TV) * 16 * MC * r);                   // projection coefficients
  b += al32(sizeof(TV) * 64 * MC);                       // B_{k-1}, Gram, R, R^{-1}
  b += al32(sizeof(double) * 32 * MC);                   // B_k, first Cholesky factor
  b += al32(sizeof(TV) * KW * NCH * 16);                 // reduction scratch
  b += al32(sizeof(int) * GI_SIZE);
  return b;
}

// Exclusive block scan of one int per thread; *total gets the sum.  Two
// __syncthreads().
template <int KT>
__device__ __forceinline__ int block_scan_excl(int x, int* wt, int& total) {
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int y = x;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int z = __shfl_up_sync(0xffffffffu, y, o);
    if (lane >= o) y += z;
  }
  if (lane == 31) wt[warp] = y;
  __syncthreads();
  int base = 0, tot = 0;
#pragma unroll
  for (int w = 0; w < KT / 32; ++w) {
    const int v = wt[w];
    if (w < warp) base += v;
    tot += v;
  }
  __syncthreads();
  total = tot;
  return base + y - x;
}

// Fixed-order block sum of NV values per thread; out[0..NV) (shared) gets the
// totals.  Two __syncthreads().
template <typename T, int NV, int KT>
__device__ __forceinline__ void block_sum_nv(const T (&v)[NV], T* red, T* out) {
  constexpr int NCH = (NV + 15) / 16;
  constexpr int KW = KT / 32;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
#pragma unroll
  for (int ch = 0; ch < NCH; ++ch) {
    T p[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) p[q] = ch * 16 + q < NV ? v[ch * 16 + q] : T(0);
    const T t = tbk::warp_reduce16(p, lane);
    if ((lane & 1) == 0 && ch * 16 + (lane >> 1) < NV) red[(warp * NCH + ch) * 16 + (lane >> 1)] = t;
  }
  __syncthreads();
  for (int x = threadIdx.x; x < NV; x += KT) {
    const int ch = x >> 4, q = x & 15;
    T s = 0;
    for (int w = 0; w < KW; ++w) s += red[(w * NCH + ch) * 16 + q];
    out[x] = s;
  }
  __syncthreads();
}

__device__ __forceinline__ int find_sorted(const int* cl, int nu, int b) {
  int lo = 0, hi = nu;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cl[mid] < b) lo = mid + 1; else hi = mid;
  }
  return (lo < nu && cl[lo] == b) ? lo : -1;
}

// (one CTA per SM: two CTAs of FP32 pairs at 128 registers measured slower)
template <typename TV, int MC, int KT, bool VKS>
__global__ void __launch_bounds__(KT, 1) krylov_group_kernel(const KryGArgs<TV> a) {
  constexpr int KW = KT / 32;
  constexpr int NV = 10 * MC;
  constexpr int NCH = (NV + 15) / 16;
  static_assert(MC >= 1 && MC <= GMAX, "group capacity");
  extern __shared__ __align__(32) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = a.r, NT = 4 * r;
  const size_t BS = 16 * (size_t)a.max_union;         // values per basis block (Dmax * 4)
  const int npi = MC * r > KW ? MC * r : KW;
  size_t off = 0;
  int* ub = reinterpret_cast<int*>(smem + off);      off += al32(sizeof(int) * a.ubuf);
  int* cl = reinterpret_cast<int*>(smem + off);      off += al32(sizeof(int) * a.max_union);
  int* rowptr = reinterpret_cast<int*>(smem + off);  off += al32(sizeof(int) * (a.max_union + 1));
  TV* W = reinterpret_cast<TV*>(smem + off);         off += al32(sizeof(TV) * MC * BS);
  TV* Vks = nullptr;
  if (VKS) {
    Vks = reinterpret_cast<TV*>(smem + off);
    off += al32(sizeof(TV) * MC * BS);
  }
  TV* V = a.Vg + (size_t)blockIdx.x * MC * r * BS;
  int2* lent = a.lent + (size_t)blockIdx.x * a.max_union * a.max_hnbr;
  if (a.lent_smem) {
    lent = reinterpret_cast<int2*>(smem + off);
    off += al32(sizeof(int2) * (size_t)a.max_union * a.max_hnbr);
  }
  TV* Cp = reinterpret_cast<TV*>(smem + off);        off += al32(sizeof(TV) * 16 * npi);
  TV* Cc = reinterpret_cast<TV*>(smem + off);        off += al32(sizeof(TV) * 16 * MC * r);
  TV* Bp = reinterpret_cast<TV*>(smem + off);
  TV* Gs = Bp + 16 * MC;
  TV* Rsh = Gs + 16 * MC;
  TV* Rish = Rsh + 16 * MC;                          off += al32(sizeof(TV) * 64 * MC);
  double* Bs = reinterpret_cast<double*>(smem + off);
  double* R1s = Bs + 16 * MC;                        off += al32(sizeof(double) * 32 * MC);
  TV* red = reinterpret_cast<TV*>(smem + off);       off += al32(sizeof(TV) * KW * NCH * 16);
  int* gi = reinterpret_cast<int*>(smem + off);
  const TV Es = (TV)a.Es, Ep = (TV)a.Ep;
  const TV chol_rel = sizeof(TV) == 4 ? (TV)1e-3 : (TV)1e-8;
  const double chol_abs = 1000.0 * a.defl_tol;

  for (int g = blockIdx.x; g < a.n_groups; g += gridDim.x) {
    const int q0 = a.g_off[g];
    const int mg = a.g_off[g + 1] - q0;
    // ---- members (every thread reads the same values)
    int mem[MC], nc[MC], c0[MC];
    bool bad = mg < 1 || mg > MC;
    int code = TB_ERR_INVALID_ARG, info = g;
#pragma unroll
    for (int t = 0; t < MC; ++t) {
      mem[t] = -1; nc[t] = 0; c0[t] = 0;
      if (!bad && t < mg) {
        const int i = a.g_idx[q0 + t];
        if (i < 0 || i >= a.n) {
          bad = true;
        } else {
          mem[t] = i;
          c0[t] = a.c_off[i];
          nc[t] = a.c_off[i + 1] - c0[t];
          const int deg = a.h_off[i + 1] - a.h_off[i];
          if (nc[t] < 1 || nc[t] > a.max_cluster || a.c_idx[c0[t]] != i) {
            bad = true; info = i;
          } else if (deg > a.max_hnbr) {
            bad = true; code = TB_ERR_CAPACITY; info = deg;
          }
        }
      }
    }
#pragma unroll
    if (bad) {
      if (tid == 0) {
        tbk::set_status(a.st, code, info);
#pragma unroll
        for (int t = 0; t < MC; ++t) if (mem[t] >= 0) a.colmask[mem[t]] = 0ull;
      }
      __syncthreads();
      continue;
    }
    // ---- union of the member clusters: sort the concatenation, drop repeats
    for (int q = tid; q < a.ubuf; q += KT) {
      const int t = q / a.max_cluster, s = q - t * a.max_cluster;
      int v = INT_MAX;
#pragma unroll
      for (int tt = 0; tt < MC; ++tt)
        if (tt == t && s < nc[tt]) v = a.c_idx[c0[tt] + s];
      ub[q] = v;
    }
    __syncthreads();
    for (int kk = 2; kk <= a.ubuf; kk <<= 1) {
      for (int j = kk >> 1; j > 0; j >>= 1) {
        for (int q = tid; q < a.ubuf; q += KT) {
          const int p = q ^ j;
          if (p > q) {
            const int x = ub[q], y = ub[p];
            if ((x > y) == ((q & kk) == 0)) { ub[q] = y; ub[p] = x; }
          }
        }
        __syncthreads();
      }
    }
    {
      const int E = a.ubuf / KT;          // ubuf is a multiple of KT
      const int qb = tid * E;
      int cnt = 0;
      for (int e = 0; e < E; ++e) {
        const int q = qb + e, v = ub[q];
        cnt += (v != INT_MAX && (q == 0 || ub[q - 1] != v)) ? 1 : 0;
      }
      int tot;
      int pos = block_scan_excl<KT>(cnt, gi + GI_WT, tot);
      for (int e = 0; e < E; ++e) {
        const int q = qb + e, v = ub[q];
        if (v != INT_MAX && (q == 0 || ub[q - 1] != v)) {
          if (pos < a.max_union) cl[pos] = v;
          ++pos;
        }
      }
      if (tid == 0) gi[GI_NU] = tot;
      __syncthreads();
    }
    const int nu = gi[GI_NU];
    if (nu > a.max_union) {
      if (tid == 0) {
        tbk::set_status(a.st, TB_ERR_CAPACITY, nu);
#pragma unroll
        for (int t = 0; t < MC; ++t) if (mem[t] >= 0) a.colmask[mem[t]] = 0ull;
      }
      __syncthreads();
      continue;
    }
    const int D = 4 * nu;
    if (tid < mg) gi[GI_SLOT + tid] = find_sorted(cl, nu, a.g_idx[q0 + tid]);
    // ---- local sparsity of H_u: counts, block-wide exclusive scan, fill
    for (int s = tid; s < nu; s += KT) {
      const int at = cl[s];
      int cnt = 0;
      const int pe = min(a.h_off[at + 1], a.h_off[at] + a.max_hnbr);
      for (int p = a.h_off[at]; p < pe; ++p) cnt += find_sorted(cl, nu, a.h_idx[p]) >= 0;
      rowptr[s] = cnt;
    }
    __syncthreads();
    {
      int v[4], tot4 = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = tid * 4 + q;
        v[q] = idx < nu ? rowptr[idx] : 0;
        tot4 += v[q];
      }
      int total;
      int run = block_scan_excl<KT>(tot4, gi + GI_WT, total);
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = tid * 4 + q;
        if (idx < nu) {
          rowptr[idx] = run;
          run += v[q];
          if (idx == nu - 1) rowptr[nu] = run;
        }
      }
      __syncthreads();
    }
    for (int s = tid; s < nu; s += KT) {
      const int at = cl[s];
      int e = rowptr[s];
      const int pe = min(a.h_off[at + 1], a.h_off[at] + a.max_hnbr);
      for (int p = a.h_off[at]; p < pe; ++p) {
        const int t = find_sorted(cl, nu, a.h_idx[p]);
        if (t >= 0) lent[e++] = make_int2(t, p);
      }
    }
    // ---- seed blocks V_{t,1} = E_{i_t}; per-target state
#pragma unroll
    for (int t = 0; t < MC; ++t) {
      if (t >= mg) continue;
      const int slot = gi[GI_SLOT + t];
      TV* V1 = V + (size_t)t * r * BS;
      for (int q = tid; q < D * 4; q += KT) {
        const int row = q >> 2, c = q & 3;
        V1[q] = (row == 4 * slot + c) ? (TV)1 : (TV)0;
      }
    }
    if (tid < 16 * MC) Bp[tid] = (TV)0;
    if (tid < MC) {
      gi[GI_MASK + 2 * tid] = tid < mg ? 0xF : 0;
      gi[GI_MASK + 2 * tid + 1] = 0;
      gi[GI_ACT + tid] = 0xF;
      gi[GI_NB + tid] = 1;
      gi[GI_LT + tid] = tid;
    }
    if (tid == 0) {
      gi[GI_LIVE] = (1 << mg) - 1;
      gi[GI_NL] = mg;
    }
    __syncthreads();
    if (tid < mg) {
      const int i = a.g_idx[q0 + tid], s = gi[GI_SLOT + tid];
      if (s < 0 || rowptr[s + 1] - rowptr[s] != a.h_off[i + 1] - a.h_off[i])
        tbk::set_status(a.st, TB_ERR_INVALID_ARG, i);
    }

    for (int k = 0; k < r; ++k) {
      const int live = gi[GI_LIVE];
      const int nl = gi[GI_NL];
      if constexpr (VKS) {               // the sweep reads V_k rows many times: stage them
        for (int q = tid; q < MC * D; q += KT) {
          const int t = q / D, row = q - t * D;
          if ((live >> t) & 1)
            st4(Vks + t * BS + row * 4, ld4(V + ((size_t)t * r + k) * BS + row * 4));
        }
        __syncthreads();
      }
      // ---- W_t = H_u V_{t,k} - V_{t,k-1} B_{t,k-1}^T for every live target;
      // item (s, alpha) = one row of every W_t, each H block read once
      for (int it = tid; it < D; it += KT) {
        const int s = it >> 2, al = it & 3;
        const TV on = al == 0 ? Es : Ep;
        TV acc[MC][4];
#pragma unroll
        for (int t = 0; t < MC; ++t) {
          const TV* Vt = VKS ? Vks + t * BS : V + ((size_t)t * r + k) * BS;
          vec4<TV> vs;
          if ((live >> t) & 1) vs = ld4(Vt + it * 4);
          else vs.v[0] = vs.v[1] = vs.v[2] = vs.v[3] = (TV)0;
#pragma unroll
          for (int c = 0; c < 4; ++c) acc[t][c] = on * vs.v[c];
        }
        const int e1 = rowptr[s + 1];
#pragma unroll 2
        for (int e = rowptr[s]; e < e1; ++e) {
          const int2 en = lent[e];
          const vec4<TV> h = hrow<TV>(a, en.y, al);
#pragma unroll
          for (int t = 0; t < MC; ++t) {
            if (!((live >> t) & 1)) continue;
            const TV* Vt = VKS ? Vks + t * BS : V + ((size_t)t * r + k) * BS;
#pragma unroll
            for (int be = 0; be < 4; ++be) {
              const vec4<TV> vt = ld4(Vt + (4 * en.x + be) * 4);
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[t][c] += h.v[be] * vt.v[c];
            }
          }
        }
#pragma unroll
        for (int t = 0; t < MC; ++t) {
          if (!((live >> t) & 1)) continue;
          if (k > 0) {
            const vec4<TV> vp = ld4(V + ((size_t)t * r + k - 1) * BS + it * 4);
            const TV* bp = Bp + t * 16;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              acc[t][c] -= vp.v[0] * bp[c * 4 + 0] + vp.v[1] * bp[c * 4 + 1] +
                           vp.v[2] * bp[c * 4 + 2] + vp.v[3] * bp[c * 4 + 3];
          }
          vec4<TV> o;
#pragma unroll
          for (int c = 0; c < 4; ++c) o.v[c] = acc[t][c];
          st4(W + t * BS + it * 4, o);
        }
      }
      __syncthreads();
      // ---- classical Gram-Schmidt per target (pass 0 yields A_k)
      const int passes = (k == r - 1) ? 1 : a.reorth_passes;
      TV gg[NV];                            // Gram partials of every final W_t
#pragma unroll
      for (int q = 0; q < NV; ++q) gg[q] = (TV)0;
      for (int pass = 0; pass < passes; ++pass) {
        const bool full = a.reorth_every <= 1 || (k % a.reorth_every) == a.reorth_every - 1;
        const int b0 = (k == r - 1) ? k : (full ? 0 : (k > 0 ? k - 1 : 0));
        const int nb = k + 1 - b0;
        const int P = nl * nb;
        const int nseg = P >= KW ? 1 : KW / P;
        const int items = P * nseg;
        for (int w = warp; w < items; w += KW) {
          const int pi = w / nseg, seg = w - pi * nseg;
          const int t = gi[GI_LT + pi / nb], b = b0 + pi % nb;
          const int rlo = (D * seg) / nseg, rhi = (D * (seg + 1)) / nseg;
          const TV* Vb = V + ((size_t)t * r + b) * BS;
          const TV* Wt = W + t * BS;
          TV acc[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) acc[q] = (TV)0;
#pragma unroll 4
          for (int row = rlo + lane; row < rhi; row += 32) {
            const vec4<TV> v = ld4(Vb + row * 4);
            const vec4<TV> x = ld4(Wt + row * 4);
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
              for (int c = 0; c < 4; ++c) acc[ii * 4 + c] += v.v[ii] * x.v[c];
          }
          const TV tot = tbk::warp_reduce16(acc, lane);
          if ((lane & 1) == 0) Cp[w * 16 + (lane >> 1)] = tot;
        }
        __syncthreads();
        for (int x = tid; x < P * 16; x += KT) {
          const int pi = x >> 4, q = x & 15;
          const int t = gi[GI_LT + pi / nb], b = b0 + pi % nb;
          TV sum = (TV)0;
          for (int sg = 0; sg < nseg; ++sg) sum += Cp[(pi * nseg + sg) * 16 + q];
          Cc[((size_t)t * r + b) * 16 + q] = sum;
        }
        __syncthreads();
        if (pass == 0 && tid < 16 * MC) {
          const int t = tid >> 4, ii = (tid >> 2) & 3, c = tid & 3;
          if ((live >> t) & 1) {
            const TV* ck = Cc + ((size_t)t * r + k) * 16;
            a.T[(size_t)a.g_idx[q0 + t] * tc_doubles(r) + 32 * k + 4 * ii + c] =
                0.5 * ((double)ck[ii * 4 + c] + (double)ck[c * 4 + ii]);     // A_k
          }
        }
        if (k == r - 1) break;
        const bool last = pass == passes - 1;
        for (int row = tid; row < D; row += KT) {
#pragma unroll
          for (int t = 0; t < MC; ++t) {
            if (!((live >> t) & 1)) continue;
            vec4<TV> x = ld4(W + t * BS + row * 4);
            for (int b = b0; b <= k; ++b) {
              const vec4<TV> v = ld4(V + ((size_t)t * r + b) * BS + row * 4);
              const TV* cb = Cc + ((size_t)t * r + b) * 16;
#pragma unroll
              for (int ii = 0; ii < 4; ++ii) {
                const vec4<TV> crow = ld4(cb + ii * 4);
#pragma unroll
                for (int c = 0; c < 4; ++c) x.v[c] -= v.v[ii] * crow.v[c];
              }
            }
            st4(W + t * BS + row * 4, x);
            if (last) {
              int q = 0;
#pragma unroll
              for (int c = 0; c < 4; ++c)
#pragma unroll
                for (int e = c; e < 4; ++e) gg[t * 10 + q++] += x.v[c] * x.v[e];
            }
          }
        }
        if (!last) __syncthreads();         // the Gram reduction below synchronises
      }
      if (k == r - 1) break;
      // ---- in-block QR per target: Cholesky QR (once when well conditioned,
      // else twice); modified Gram-Schmidt when a pivot refuses
      int pend = live;
      for (int cq = 0; cq < 2; ++cq) {
        block_sum_nv<TV, NV, KT>(gg, red, Gs);
        if (tid < MC && ((pend >> tid) & 1)) {
          const int t = tid;
          TV G[16];
          int q = 0;
#pragma unroll
          for (int c = 0; c < 4; ++c)
#pragma unroll
            for (int e = c; e < 4; ++e) {
              G[c * 4 + e] = Gs[t * 10 + q];
              G[e * 4 + c] = Gs[t * 10 + q];
              ++q;
            }
          TV R[16], Ri[16];
          bool well;
          const bool ok = chol4(G, R, chol_rel, cq == 0 ? chol_abs : 0.0, well);
          triinv4(R, Ri);
#pragma unroll
          for (int q2 = 0; q2 < 16; ++q2) { Rsh[t * 16 + q2] = R[q2]; Rish[t * 16 + q2] = Ri[q2]; }
          const int okf = ok ? ((cq == 0 && well && sizeof(TV) == 4) ? 2 : 1) : 0;
          gi[GI_OK + t] = okf;
          if (cq == 0) gi[GI_CS + t] = 0;
          if (!okf) {
            gi[GI_CS + t] = cq + 1;
          } else if (okf == 2) {            // B_k = R1, done
#pragma unroll
            for (int q2 = 0; q2 < 16; ++q2) Bs[t * 16 + q2] = (double)R[q2];
            gi[GI_ACT + t] = 0xF;
          } else if (cq == 0) {
#pragma unroll
            for (int q2 = 0; q2 < 16; ++q2) R1s[t * 16 + q2] = (double)R[q2];
          } else {                          // B_k = R2 R1
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                double s = 0.0;
#pragma unroll
                for (int j = 0; j < 4; ++j) s += (double)R[rr * 4 + j] * R1s[t * 16 + j * 4 + c];
                Bs[t * 16 + rr * 4 + c] = s;
              }
            gi[GI_ACT + t] = 0xF;
          }
        }
        __syncthreads();
        int app = 0, two = 0;
#pragma unroll
        for (int t = 0; t < MC; ++t) {
          if (!((pend >> t) & 1)) continue;
          const int o = gi[GI_OK + t];
          if (o) app |= 1 << t;
          if (cq == 0 && o == 1) two |= 1 << t;
        }
#pragma unroll
        for (int q = 0; q < NV; ++q) gg[q] = (TV)0;
        if (app) {
          for (int row = tid; row < D; row += KT) {
#pragma unroll
            for (int t = 0; t < MC; ++t) {
              if (!((app >> t) & 1)) continue;
              const vec4<TV> x = ld4(W + t * BS + row * 4);
              const TV* Ri = Rish + t * 16;
              vec4<TV> y;
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                TV s = (TV)0;
#pragma unroll
                for (int j = 0; j <= c; ++j) s += x.v[j] * Ri[j * 4 + c];
                y.v[c] = s;
              }
              const bool again = (two >> t) & 1;
              TV* dst = again ? W + t * BS : V + ((size_t)t * r + k + 1) * BS;
              st4(dst + row * 4, y);
              if (again) {
                int q = 0;
#pragma unroll
                for (int c = 0; c < 4; ++c)
#pragma unroll
                  for (int e = c; e < 4; ++e) gg[t * 10 + q++] += y.v[c] * y.v[e];
              }
            }
          }
        }
        pend = two;
        if (pend == 0) break;
      }
      __syncthreads();
      int mgs = 0;
#pragma unroll
      for (int t = 0; t < MC; ++t)
        if (((live >> t) & 1) && gi[GI_CS + t] != 0) mgs |= 1 << t;
      if (mgs) {
        if (warp < MC && ((mgs >> warp) & 1)) {
          const int t = warp;
          TV* Wt = W + t * BS;
          TV* Vn = V + ((size_t)t * r + k + 1) * BS;
          const int cs = gi[GI_CS + t];
          double R[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) R[q] = 0.0;
          int act = 0;
          bool nonfinite = false;
#pragma unroll
          for (int c = 0; c < 4; ++c) {
            for (int pass = 0; pass < 2; ++pass) {
              if (c == 0) break;
              TV dd[3] = {(TV)0, (TV)0, (TV)0};
              for (int row = lane; row < D; row += 32) {
                const TV w = Wt[row * 4 + c];
#pragma unroll
                for (int j = 0; j < 3; ++j) if (j < c) dd[j] += Vn[row * 4 + j] * w;
              }
#pragma unroll
              for (int j = 0; j < 3; ++j) if (j < c) dd[j] = tbk::warp_sum(dd[j]);
              for (int row = lane; row < D; row += 32) {
                TV w = Wt[row * 4 + c];
#pragma unroll
                for (int j = 0; j < 3; ++j) if (j < c) w -= dd[j] * Vn[row * 4 + j];
                Wt[row * 4 + c] = w;
              }
#pragma unroll
              for (int j = 0; j < 3; ++j) if (j < c) R[j * 4 + c] += (double)dd[j];
            }
            TV nn = (TV)0;
            for (int row = lane; row < D; row += 32) {
              const TV w = Wt[row * 4 + c];
              nn += w * w;
            }
            nn = tbk::warp_sum(nn);
            const double nrm = sqrt((double)nn);
            if (!isfinite(nrm)) nonfinite = true;
            if (nrm > a.defl_tol) {
              const TV inv = (TV)(1.0 / nrm);
              for (int row = lane; row < D; row += 32) Vn[row * 4 + c] = Wt[row * 4 + c] * inv;
              R[c * 4 + c] = nrm;
              act |= 1 << c;
            } else {
              for (int row = lane; row < D; row += 32) Vn[row * 4 + c] = (TV)0;
            }
          }
          if (lane == 0) {
            if (cs == 2) {              // W was already W R1^{-1}: B_k = R_mgs R1
#pragma unroll
              for (int rr = 0; rr < 4; ++rr)
#pragma unroll
                for (int c = 0; c < 4; ++c) {
                  double s = 0.0;
#pragma unroll
                  for (int j = 0; j < 4; ++j) s += R[rr * 4 + j] * R1s[t * 16 + j * 4 + c];
                  Bs[t * 16 + rr * 4 + c] = s;
                }
            } else {
#pragma unroll
              for (int q = 0; q < 16; ++q) Bs[t * 16 + q] = R[q];
            }
            gi[GI_ACT + t] = act;
            if (nonfinite) tbk::set_status(a.st, TB_ERR_NONFINITE, a.g_idx[q0 + t]);
          }
        }
        __syncthreads();
      }
      if (tid < MC && ((live >> tid) & 1)) {
        const int t = tid;
        const int i = a.g_idx[q0 + t];
        double* Ti = a.T + (size_t)i * tc_doubles(r);
        const int act = gi[GI_ACT + t];
        const double* bs = Bs + t * 16;
#pragma unroll
        for (int q = 0; q < 16; ++q) Ti[32 * k + 16 + q] = bs[q];              // B_k
        unsigned long long mask = ((unsigned long long)(unsigned)gi[GI_MASK + 2 * t + 1] << 32) |
                                  (unsigned)gi[GI_MASK + 2 * t];
        mask |= (unsigned long long)act << (4 * (k + 1));
        gi[GI_MASK + 2 * t] = (int)(mask & 0xffffffffull);
        gi[GI_MASK + 2 * t + 1] = (int)(mask >> 32);
        if (!isfinite(bs[0] + bs[5] + bs[10] + bs[15])) tbk::set_status(a.st, TB_ERR_NONFINITE, i);
      }
      if (tid < 16 * MC && ((live >> (tid >> 4)) & 1)) Bp[tid] = (TV)Bs[tid];
      __syncthreads();
      if (tid == 0) {
        int live2 = 0, nl2 = 0;
        for (int t = 0; t < MC; ++t) {
          if (!((live >> t) & 1) || gi[GI_ACT + t] == 0) continue;
          live2 |= 1 << t;
          gi[GI_NB + t] = k + 2;
          gi[GI_LT + nl2++] = t;
        }
        gi[GI_LIVE] = live2;
        gi[GI_NL] = nl2;
      }
      __syncthreads();
      if (gi[GI_LIVE] == 0) break;
    }
    // ---- outputs per target: column mask, rows of V for it and its H neighbours
    for (int t = 0; t < mg; ++t) {
      const int i = a.g_idx[q0 + t];
      const int slot = gi[GI_SLOT + t], nbk = gi[GI_NB + t];
      if (tid == 0)
        a.colmask[i] = ((unsigned long long)(unsigned)gi[GI_MASK + 2 * t + 1] << 32) |
                       (unsigned)gi[GI_MASK + 2 * t];
      const int deg = a.h_off[i + 1] - a.h_off[i];
      const size_t ybase = (size_t)(i + a.h_off[i]) * 4;
      const int nrows = (deg + 1) * 4;
      const TV* Vt = V + (size_t)t * r * BS;
      // (a row with fewer entries than the H list was reported above; its
      // missing neighbours get zero rows)
      const int rcnt = slot >= 0 ? rowptr[slot + 1] - rowptr[slot] : 0;
      for (int q = tid; q < nrows * NT; q += KT) {
        const int rr = q / NT, col = q - rr * NT;
        const int qq = rr >> 2, beta = rr & 3;
        const int sl = qq == 0 ? slot : (qq - 1 < rcnt ? lent[rowptr[slot] + qq - 1].x : -1);
        const int b = col >> 2, c = col & 3;
        TV val = (TV)0;
        if (b < nbk && sl >= 0) val = Vt[(size_t)b * BS + (4 * sl + beta) * 4 + c];
        a.Y[(ybase + rr) * NT + col] = val;
      }
    }
    __syncthreads();
  }
}

int pow2_at_least(int x) {
  int p = 1;
  while (p < x) p <<= 1;
  return p;
}

template <typename TV, int MC, int KT, bool VKS>
tb_status kryg_configure_t(tb_ctx* c, int max_smem) {
  const tb_params& p = c->p;
  const int mu = c->grp_max_union;
  if (mu > 4 * KT) return TB_ERR_CAPACITY;                 // block scan: 4 slots per thread
  int ubuf = pow2_at_least(MC * p.max_cluster);
  if (ubuf < KT) ubuf = KT;
  if (ubuf > UBUF_MAX) return TB_ERR_CAPACITY;
  const size_t b0 = kryg_smem_bytes<TV, MC, KT, VKS>(p.r, mu, p.max_hnbr, false, ubuf);
  const size_t b1 = kryg_smem_bytes<TV, MC, KT, VKS>(p.r, mu, p.max_hnbr, true, ubuf);
  if ((int)b0 > max_smem) return TB_ERR_CAPACITY;
  const bool lsmem = (int)b1 <= max_smem;
  const size_t bytes = lsmem ? b1 : b0;
  TB_CUDA_TRY(cudaFuncSetAttribute(krylov_group_kernel<TV, MC, KT, VKS>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  int occ = 0;
  TB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(
      &occ, krylov_group_kernel<TV, MC, KT, VKS>, KT, bytes));
  if (occ < 1) return TB_ERR_CAPACITY;
  c->grp_mc = MC;
  c->grp_threads = KT;
  c->grp_vks = VKS;
  c->grp_lsmem = lsmem;
  c->grp_smem = bytes;
  c->grp_ubuf = ubuf;
  c->grp_grid = c->num_sms * occ;
  return TB_OK;
}

template <typename TV, int MC, int KT, bool VKS>
tb_status kryg_launch_t(tb_ctx* c, int n, int n_groups, const int* g_off, const int* g_idx,
                        const int* c_off, const int* c_idx, const int* h_off, const int* h_idx,
                        const TV* H, const float* Hsk, cudaStream_t s) {
  const tb_params& p = c->p;
  KryGArgs<TV> a;
  a.Hsk = reinterpret_cast<const float4*>(Hsk);
  a.Vss = (float)p.Vss; a.Vsp = (float)p.Vsp; a.Cpp = (float)(p.Vpps - p.Vppp);
  a.Vppp = (float)p.Vppp;
  a.n = n; a.n_groups = n_groups; a.r = p.r; a.max_cluster = p.max_cluster;
  a.max_union = c->grp_max_union; a.max_hnbr = p.max_hnbr;
  a.reorth_passes = p.reorth_passes; a.reorth_every = p.reorth_every; a.ubuf = c->grp_ubuf;
  a.Es = p.Es; a.Ep = p.Ep; a.defl_tol = p.defl_tol;
  a.g_off = g_off; a.g_idx = g_idx; a.c_off = c_off; a.c_idx = c_idx;
  a.h_off = h_off; a.h_idx = h_idx; a.H = H;
  a.T = c->T; a.Y = reinterpret_cast<TV*>(c->Y); a.colmask = c->colmask;
  a.Vg = reinterpret_cast<TV*>(c->grp_V); a.lent = c->grp_lent;
  a.lent_smem = c->grp_lsmem ? 1 : 0; a.st = c->d_status;
  const int grid = n_groups < c->grp_grid ? n_groups : c->grp_grid;
  if (grid <= 0) return TB_OK;
  krylov_group_kernel<TV, MC, KT, VKS><<<grid, KT, c->grp_smem, s>>>(a);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}

template <typename TV, int MC>
tb_status kryg_configure_mc(tb_ctx* c, int max_smem, int kt, bool nostage) {
  if (kt == 512) {
    if (!nostage && kryg_configure_t<TV, MC, 512, true>(c, max_smem) == TB_OK) return TB_OK;
    if (kryg_configure_t<TV, MC, 512, false>(c, max_smem) == TB_OK) return TB_OK;
  }
  if (!nostage && kryg_configure_t<TV, MC, 256, true>(c, max_smem) == TB_OK) return TB_OK;
  return kryg_configure_t<TV, MC, 256, false>(c, max_smem);
}

}  // namespace

int group_grid_cells(int n, int m) {
  int g = 1;
  while (g < 1024 && (long long)m * (g + 1) * (g + 1) * (g + 1) <= (long long)n) ++g;
  return g;
}

tb_status krylov_group_configure(tb_ctx* c) {
  const tb_params& p = c->p;
  c->grp_max_union = p.max_union > 0 ? p.max_union
                                     : (p.group_m * p.max_cluster < tbk::MAX_CLUSTER
                                            ? p.group_m * p.max_cluster : tbk::MAX_CLUSTER);
  int dev = 0, max_smem = 0;
  TB_CUDA_TRY(cudaGetDevice(&dev));
  TB_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  // 512 threads for groups of up to four in FP32 (the FP64 kernel would
  // spill at 128 registers), else 256; the staged copy of V_k when it fits.
  const int kt = (p.group_m > 2 && p.prec != TB_PREC_FP64) ? 512 : 256;
  const bool nostage = false;
  if (p.prec == TB_PREC_FP64)
    return p.group_m > 2 ? kryg_configure_mc<double, 4>(c, max_smem, kt, nostage)
                         : kryg_configure_mc<double, 2>(c, max_smem, kt, nostage);
  return p.group_m > 2 ? kryg_configure_mc<float, 4>(c, max_smem, kt, nostage)
                       : kryg_configure_mc<float, 2>(c, max_smem, kt, nostage);
}

size_t krylov_group_basis_bytes(const tb_ctx* c) {
  if (c->grp_grid <= 0) return 0;
  const size_t tv = c->p.prec == TB_PREC_FP64 ? sizeof(double) : sizeof(float);
  return (size_t)c->grp_grid * c->grp_mc * c->p.r * 16 * (size_t)c->grp_max_union * tv;
}

tb_status launch_group_atoms(tb_ctx* c, int n, const double* pos, double L, int* g_off,
                             int* g_idx, cudaStream_t s) {
  const int m = c->p.group_m;
  const int g = group_grid_cells(n, m);
  TB_CUDA_TRY(cudaMemsetAsync(c->grp_cnt, 0, sizeof(int) * (size_t)n, s));
  const int bx = (n + 255) / 256;
  int split = (2 * c->num_sms + bx - 1) / bx;
  if (split < 1) split = 1;
  if (split > 64) split = 64;
  const int per = (n + split - 1) / split;
  split = (n + per - 1) / per;
  group_count_kernel<<<dim3(bx, split), 256, 0, s>>>(n, pos, L, g, per, c->grp_cnt);
  TB_CUDA_TRY(cudaGetLastError());
  group_scatter_kernel<<<(n + 1 + 255) / 256, 256, 0, s>>>(n, m, c->grp_cnt, g_off, g_idx);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}

tb_status launch_krylov_grouped(tb_ctx* c, int n, int n_groups, const int* g_off,
                                const int* g_idx, const int* c_off, const int* c_idx,
                                const int* h_off, const int* h_idx, const double* Hblk,
                                const float* Hsk, cudaStream_t s) {
#define TB_KRYG_DISPATCH(TV, MC, H)                                                             \
  do {                                                                                          \
    if (c->grp_threads == 512)                                                                  \
      return c->grp_vks ? kryg_launch_t<TV, MC, 512, true>(c, n, n_groups, g_off, g_idx, c_off, \
                                                           c_idx, h_off, h_idx, H, Hsk, s)           \
                        : kryg_launch_t<TV, MC, 512, false>(c, n, n_groups, g_off, g_idx,       \
                                                            c_off, c_idx, h_off, h_idx, H, Hsk, s);  \
    return c->grp_vks ? kryg_launch_t<TV, MC, 256, true>(c, n, n_groups, g_off, g_idx, c_off,   \
                                                         c_idx, h_off, h_idx, H, Hsk, s)             \
                      : kryg_launch_t<TV, MC, 256, false>(c, n, n_groups, g_off, g_idx, c_off,  \
                                                          c_idx, h_off, h_idx, H, Hsk, s);           \
  } while (0)
  if (c->grp_grid <= 0) return TB_ERR_INVALID_ARG;
  if (c->p.prec == TB_PREC_FP64) {
    if (c->grp_mc == 4) TB_KRYG_DISPATCH(double, 4, Hblk);
    TB_KRYG_DISPATCH(double, 2, Hblk);
  }
  if (!Hsk) return TB_ERR_INVALID_ARG;
  const float* none = nullptr;
  if (c->grp_mc == 4) TB_KRYG_DISPATCH(float, 4, none);
  TB_KRYG_DISPATCH(float, 2, none);
#undef TB_KRYG_DISPATCH
}
