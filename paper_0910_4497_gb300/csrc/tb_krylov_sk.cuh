// Block Lanczos of one target atom for the mixed path (Sec. 3, Eq. (Krylov)
// and the block form of Eqs. (lanczos) / (lanczos_blas3)), on the cluster
// Hamiltonian H_c of Sec. 2 given as Slater-Koster records.
//
// The 4x4 block of a directed bond i -> j is fixed by the distance scaling
// s(|d|) and the direction l = d/|d| (d = R_j - R_i) through the table of
// Eq. (1); the sweep applies it to a 4-vector u = (u_s, u_p) without forming
// it:
//   (H u)_s = s [Vss u_s + Vsp (l.u_p)]
//   (H u)_p = l s [(Vpps - Vppp)(l.u_p) - Vsp u_s] + s Vppp u_p
// so a target's in-cluster bonds cost one 16-byte record each (8 bytes in
// BF16), staged in shared memory once per target, instead of a 64-byte block
// read from L2 in every sweep.
//
// Layout: every block of the Krylov basis (and W) is stored slot-major with
// the 4x4 block of cluster slot s transposed, [s][c][b] = V[4s + b][c], so
// that one thread per (slot s, column c) reads the neighbour's column c as
// one float4.  Items are (s, c) = 4s + c; the four columns of a slot are
// neighbouring lanes of one warp.  Within slot s, column c sits at position
// c ^ ((s >> 1) & 3): lanes reading one column of consecutive slots (one slot
// per lane, or four lanes per slot) then hit distinct shared-memory banks,
// which the plain 16-float pitch does not give (every other slot on the same
// banks).
//
// Per step k (V_k, V_{k-1} and W rotate through three shared-memory buffers;
// every block is also written to the CTA's basis slot in global memory for
// the full reorthogonalisations and the output rows):
//   W = H_c V_k - V_{k-1} B_{k-1}^T              sweep
//   C = Q^T W, W -= Q C                          classical Gram-Schmidt against
//                                                Q = [V_b0..V_k] (all blocks every
//                                                reorth_every steps, else the last
//                                                two); the V_k part of C is A_k
//   W = V_{k+1} B_k                               Cholesky QR (twice unless the
//                                                first factor shows a well-
//                                                conditioned block), modified
//                                                Gram-Schmidt with deflation
//                                                when a pivot is refused
// T is written compactly: per target the 2r - 1 blocks A_0, B_0, A_1, ...
#pragma once
#include <cuda_bf16.h>
#include <type_traits>
#include "tb_internal.cuh"
#include "tb_krylov_common.cuh"

namespace tbsk {

using namespace tbkry;

constexpr int KT = 128;                 // threads per target
constexpr int KW = KT / 32;
constexpr int SP = 16;                  // floats per cluster slot in a basis block
constexpr int SPB = 4;                  // BF16 copy of V_k: 8-byte words per slot
constexpr int HC = 3 * SP;              // cached neighbour slots per slot during set-up

// Offset (floats) of column c of cluster slot s in a basis block:
// (SP s | 4 f(s)) ^ 4c with f(s) = (s >> 1) & 3; the first part is what the
// local sparsity stores per neighbour, so a lane finds its column with one XOR.
__host__ __device__ __forceinline__ int sbase(int s) { return SP * s + 4 * ((s >> 1) & 3); }
__host__ __device__ __forceinline__ int cofs(int s, int c) { return sbase(s) ^ (4 * c); }
constexpr int FL_MASK = 0, FL_ACT = 2, FL_OK = 3;   // flags[4..8): scan scratch

struct SkArgs {
  int n, r, max_cluster, max_hnbr, reorth_passes, reorth_every;
  int ecap;                             // local entries kept in shared memory
  float Es, Ep, Vss, Vsp, Cpp, Vppp;    // Cpp = Vpps - Vppp
  double defl_tol;
  const int* c_off;
  const int* c_idx;
  const int* h_off;
  const int* h_idx;
  const float4* Hsk;                    // (s, l_x, l_y, l_z) per directed bond
  double* T;                            // compact block tridiagonal, tc_doubles(r) per target
  float* Y;
  unsigned long long* colmask;
  float* Vg;                            // per-CTA basis slots: r blocks of 16 max_cluster
  int2* bref;                           // per-CTA overflow (max_cluster * max_hnbr entries):
                                        //   bond index and neighbour offset of each local entry
  int* st;
};

__host__ __device__ __forceinline__ size_t al32(size_t x) { return (x + 31) & ~size_t(31); }

template <bool BF>
__host__ __device__ inline size_t sk_rec_bytes() { return BF ? 8 : 16; }

// Shared memory of one target (bytes).
template <bool BF>
__host__ __device__ inline size_t sk_smem_bytes(int r, int max_cluster, int ecap) {
  const size_t MC = (size_t)max_cluster;
  size_t b = 0;
  b += al32(sizeof(int) * MC);                       // cl
  b += al32(sizeof(int) * (MC + 1));                 // roff
  b += al32(sizeof(float) * 3 * SP * MC);            // V_k, V_{k-1}, W
  if (BF) b += al32(sizeof(uint2) * SPB * MC);       // BF16 copy of V_k for the sweep
  b += al32(sk_rec_bytes<BF>() * (size_t)ecap);      // records
  b += al32(sizeof(int) * (size_t)ecap);             // neighbour offsets
  const int np = r > KW ? r : KW;
  b += al32(sizeof(float) * 16 * np);                // projection partials
  b += al32(sizeof(float) * 16 * r);                 // projection coefficients
  b += al32(sizeof(float) * 16 * 3);                 // B_{k-1}, R, R^-1
  b += al32(sizeof(float) * 16 * KW);                // reduction scratch
  b += al32(sizeof(float) * 32 * KW);                // projections summed in the sweep
  b += al32(sizeof(double) * 48);                    // B_k, first Cholesky factor, MGS factor
  b += al32(sizeof(int) * 8);                        // flags
  return b;
}

__device__ __forceinline__ uint2 pack_bf16x4(float4 v) {
  const __nv_bfloat162 a = __floats2bfloat162_rn(v.x, v.y);
  const __nv_bfloat162 b = __floats2bfloat162_rn(v.z, v.w);
  return make_uint2(*reinterpret_cast<const unsigned*>(&a), *reinterpret_cast<const unsigned*>(&b));
}
__device__ __forceinline__ float4 unpack_bf16x4(uint2 u) {
  return make_float4(__uint_as_float(u.x << 16), __uint_as_float(u.x & 0xffff0000u),
                     __uint_as_float(u.y << 16), __uint_as_float(u.y & 0xffff0000u));
}

__device__ __forceinline__ float4 f4(const float* p) { return *reinterpret_cast<const float4*>(p); }
__device__ __forceinline__ void sf4(float* p, float4 v) { *reinterpret_cast<float4*>(p) = v; }
__device__ __forceinline__ float dot4(float4 a, float4 b) {
  return fmaf(a.x, b.x, fmaf(a.y, b.y, fmaf(a.z, b.z, a.w * b.w)));
}
__device__ __forceinline__ float4 axpy4(float a, float4 x, float4 y) {   // y + a x
  return make_float4(fmaf(a, x.x, y.x), fmaf(a, x.y, y.y), fmaf(a, x.z, y.z), fmaf(a, x.w, y.w));
}
__device__ __forceinline__ float comp(float4 v, int q) {
  return q == 0 ? v.x : (q == 1 ? v.y : (q == 2 ? v.z : v.w));
}

__device__ __forceinline__ int find_slot(const int* cl, int nc, int b) {
  if (b == cl[0]) return 0;
  int lo = 1, hi = nc;
  while (lo < hi) {
    const int mid = (lo + hi) >> 1;
    if (cl[mid] < b) lo = mid + 1; else hi = mid;
  }
  return (lo < nc && cl[lo] == b) ? lo : -1;
}

// Exclusive scan of v[0..m) in place (m <= 8 KT), v[m] = total; all threads.
__device__ __forceinline__ void block_scan(int* v, int m, int* wtot) {
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int per = (m + KT - 1) / KT;
  const int s0 = min(m, tid * per), s1 = min(m, s0 + per);
  int loc = 0;
  for (int s = s0; s < s1; ++s) loc += v[s];
  int inc = loc;
#pragma unroll
  for (int o = 1; o < 32; o <<= 1) {
    const int y = __shfl_up_sync(0xffffffffu, inc, o);
    if (lane >= o) inc += y;
  }
  if (lane == 31) wtot[warp] = inc;
  __syncthreads();
  int base = 0;
#pragma unroll
  for (int w = 0; w < KW; ++w) base += w < warp ? wtot[w] : 0;
  int run = base + inc - loc;
  for (int s = s0; s < s1; ++s) {
    const int t = v[s];
    v[s] = run;
    run += t;
  }
  if (tid == KT - 1) v[m] = run;
  __syncthreads();
}

// Compact T: block 2k = A_k, block 2k+1 = B_k (T[4(k+1)+j][4k+c] = B_k[j][c]).
__device__ __forceinline__ double* tc_block(double* Ti, int blk) { return Ti + 16 * blk; }

template <bool BF>
__device__ __forceinline__ void krylov_sk_target(const SkArgs& a, const int i) {
  extern __shared__ __align__(32) unsigned char smem[];
  using Rec = typename std::conditional<BF, uint2, float4>::type;
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = a.r, NT = 4 * r, MC = a.max_cluster;
  const int np = r > KW ? r : KW;
  size_t off = 0;
  int* cl = reinterpret_cast<int*>(smem + off);       off += al32(sizeof(int) * MC);
  int* roff = reinterpret_cast<int*>(smem + off);     off += al32(sizeof(int) * (MC + 1));
  float* const bufs = reinterpret_cast<float*>(smem + off);
  off += al32(sizeof(float) * 3 * SP * MC);
  uint2* vbf = nullptr;
  if (BF) { vbf = reinterpret_cast<uint2*>(smem + off); off += al32(sizeof(uint2) * SPB * MC); }
  Rec* rec_s = reinterpret_cast<Rec*>(smem + off);    off += al32(sizeof(Rec) * (size_t)a.ecap);
  int* rsl_s = reinterpret_cast<int*>(smem + off);    off += al32(sizeof(int) * (size_t)a.ecap);
  float* Cp = reinterpret_cast<float*>(smem + off);   off += al32(sizeof(float) * 16 * np);
  float* Cc = reinterpret_cast<float*>(smem + off);   off += al32(sizeof(float) * 16 * r);
  float* Bp = reinterpret_cast<float*>(smem + off);
  float* Rsh = Bp + 16;
  float* Rish = Rsh + 16;                              off += al32(sizeof(float) * 48);
  float* red = reinterpret_cast<float*>(smem + off);  off += al32(sizeof(float) * 16 * KW);
  float* Pw = reinterpret_cast<float*>(smem + off);   off += al32(sizeof(float) * 32 * KW);
  double* Bs = reinterpret_cast<double*>(smem + off);
  double* R1s = Bs + 16;
  double* Rm = Bs + 32;                               off += al32(sizeof(double) * 48);
  int* flags = reinterpret_cast<int*>(smem + off);
  float* const Vg = a.Vg + (size_t)blockIdx.x * r * SP * MC;
  const size_t VB = (size_t)SP * MC;                   // floats per basis block
  const size_t gcap = (size_t)MC * a.max_hnbr;
  const float Es = a.Es, Ep = a.Ep, Vss = a.Vss, Vsp = a.Vsp, Cpp = a.Cpp, Vppp = a.Vppp;
  const float chol_rel = 1e-3f;
  const double chol_abs = 1000.0 * a.defl_tol;
  double* const Ti = a.T + (size_t)i * tc_doubles(r);

  const int c0 = a.c_off[i];
  const int nc = a.c_off[i + 1] - c0;
  if (nc < 1 || nc > MC || a.c_idx[c0] != i) {
    if (tid == 0) {
      tbk::set_status(a.st, TB_ERR_INVALID_ARG, i);
      a.colmask[i] = 0ull;
    }
    __syncthreads();
    return;
  }
  const int deg = a.h_off[i + 1] - a.h_off[i];
  if (deg > a.max_hnbr) {
    if (tid == 0) {
      tbk::set_status(a.st, TB_ERR_CAPACITY, deg);
      a.colmask[i] = 0ull;
    }
    __syncthreads();
    return;
  }
  for (int s = tid; s < nc; s += KT) cl[s] = a.c_idx[c0 + s];
  __syncthreads();
  // ---- local sparsity of H_c: per slot, its in-cluster Hamiltonian
  // neighbours in list order (count, scan, fill), each as a record and the
  // neighbour block's offset; the records go to shared memory when they fit,
  // else to the CTA's overflow slot
  // (the neighbours' slots found in the count pass are kept for the fill pass
  // in the basis buffers, free until the seed, when the lists are short)
  int* const hsl = reinterpret_cast<int*>(bufs);
  const bool cache = a.max_hnbr <= HC;
  for (int s = tid; s < nc; s += KT) {
    const int at = cl[s];
    const int p0 = a.h_off[at];
    const int pe = min(a.h_off[at + 1], p0 + a.max_hnbr);
    int e = 0;
    for (int p = p0; p < pe; ++p) {
      const int t = find_slot(cl, nc, a.h_idx[p]);
      if (cache) hsl[s * HC + (p - p0)] = t;
      e += t >= 0;
    }
    roff[s] = e;
  }
  __syncthreads();
  block_scan(roff, nc, flags + 8 - KW);                // wtot scratch: the last flag words
  const int ne = roff[nc];
  // a target whose records do not fit keeps, per entry, the bond index in its
  // CTA's overflow slot and reads the record from the bond table (L2) in
  // every sweep
  const bool ovf = ne > a.ecap;
  Rec* const rec = rec_s;
  int* const rsl = rsl_s;
  int2* const bref = a.bref + (size_t)blockIdx.x * gcap;
  for (int s = tid; s < nc; s += KT) {
    const int at = cl[s];
    const int p0 = a.h_off[at];
    const int pe = min(a.h_off[at + 1], p0 + a.max_hnbr);
    int e = roff[s];
    for (int p = p0; p < pe; ++p) {
      const int t = cache ? hsl[s * HC + (p - p0)] : find_slot(cl, nc, a.h_idx[p]);
      if (t >= 0) {
        if (ovf) {
          bref[e] = make_int2(p, sbase(t));
        } else {
          const float4 hv = __ldg(a.Hsk + p);
          if constexpr (BF) rec[e] = pack_bf16x4(hv);
          else rec[e] = hv;
          rsl[e] = sbase(t);
        }
        ++e;
      }
    }
  }
  __syncthreads();                                     // the cache is overwritten below
  // seed block V_1 = E_i: slot 0 holds the identity
  float* Vk = bufs;
  float* Vkm1 = bufs + VB;
  float* W = bufs + 2 * VB;
  for (int q = tid; q < SP * nc; q += KT) {
    const float v = (q < 16 && (q >> 2) == (q & 3)) ? 1.f : 0.f;
    Vk[q] = v;
    Vg[q] = v;
  }
  if constexpr (BF) {
    for (int q = tid; q < 4 * nc; q += KT) {
      const int sl = q >> 2, c = q & 3;
      vbf[SPB * sl + c] = pack_bf16x4(make_float4(sl == 0 && c == 0 ? 1.f : 0.f,
                                                   sl == 0 && c == 1 ? 1.f : 0.f,
                                                   sl == 0 && c == 2 ? 1.f : 0.f,
                                                   sl == 0 && c == 3 ? 1.f : 0.f));
    }
  }
  if (tid < 16) Bp[tid] = 0.f;
  if (tid == 0) { flags[FL_MASK] = 0xF; flags[FL_MASK + 1] = 0; flags[FL_ACT] = 0xF; }
  __syncthreads();
  if (tid == 0 && roff[1] - roff[0] != deg) tbk::set_status(a.st, TB_ERR_INVALID_ARG, i);

  const int D4 = 4 * nc;                 // items (slot, column)
  int nblocks = 1;
  for (int k = 0; k < r; ++k) {
    // ---- W = H_c V_k - V_{k-1} B_{k-1}^T, item (s, c).  The projections of
    // W on V_k and V_{k-1} (the first classical Gram-Schmidt pass for these
    // two blocks) are summed here from the slot's blocks, which the item has
    // at hand: pk[ii] = sum (V_k)[., ii] W[., c], pm likewise for V_{k-1}.
    float pk[4] = {0.f, 0.f, 0.f, 0.f}, pm[4] = {0.f, 0.f, 0.f, 0.f};
    for (int it = tid; it < D4; it += KT) {
      const int s = it >> 2, c = it & 3, c4x = 4 * c;
      const float4 u0 = f4(Vk + cofs(s, c));
      float4 acc = make_float4(Es * u0.x, Ep * u0.y, Ep * u0.z, Ep * u0.w);
      // one term of (H_c u)_s from the bond record hv = (s(r), l) and the
      // neighbour's column u
      auto term = [&](const float4 hv, const float4 u) {
        const float dt = fmaf(hv.y, u.y, fmaf(hv.z, u.z, hv.w * u.w));
        const float ps = fmaf(Vss, u.x, Vsp * dt);
        const float pp = fmaf(Cpp, dt, -Vsp * u.x);
        acc.x = fmaf(hv.x, ps, acc.x);
        const float t = hv.x * pp, w = hv.x * Vppp;
        acc.y = fmaf(hv.y, t, fmaf(w, u.y, acc.y));
        acc.z = fmaf(hv.z, t, fmaf(w, u.z, acc.z));
        acc.w = fmaf(hv.w, t, fmaf(w, u.w, acc.w));
      };
      // column c of the neighbour block at offset o (slot-major, swizzled)
      auto col = [&](const int o) -> float4 {
        if constexpr (BF) return unpack_bf16x4(vbf[((o >> 2) & ~3) + c]);   // SPB * slot
        else return f4(Vk + (o ^ c4x));
      };
      int e = roff[s];
      const int e1 = roff[s + 1];
      if (ovf) {
        // records gathered from the bond table (L2): the loads of four
        // entries are issued before their arithmetic
        for (; e + 4 <= e1; e += 4) {
          int2 q[4];
          float4 hv[4];
#pragma unroll
          for (int j = 0; j < 4; ++j) q[j] = bref[e + j];
#pragma unroll
          for (int j = 0; j < 4; ++j) hv[j] = __ldg(a.Hsk + q[j].x);
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            if constexpr (BF) hv[j] = unpack_bf16x4(pack_bf16x4(hv[j]));
            term(hv[j], col(q[j].y));
          }
        }
        for (; e < e1; ++e) {
          const int2 q = bref[e];
          float4 hv = __ldg(a.Hsk + q.x);
          if constexpr (BF) hv = unpack_bf16x4(pack_bf16x4(hv));
          term(hv, col(q.y));
        }
      } else {
#pragma unroll 2
        for (; e < e1; ++e) {
          float4 hv;
          if constexpr (BF) hv = unpack_bf16x4(rec[e]);
          else hv = rec[e];
          term(hv, col(rsl[e]));
        }
      }
      float4 vm[4];
      if (k > 0) {
        const float4 b = f4(Bp + 4 * c);            // B_{k-1}[c][d], d >= c
#pragma unroll
        for (int d = 0; d < 4; ++d) {
          vm[d] = f4(Vkm1 + cofs(s, d));
          if (d >= c) acc = axpy4(-comp(b, d), vm[d], acc);
        }
      }
      sf4(W + cofs(s, c), acc);
#pragma unroll
      for (int ii = 0; ii < 4; ++ii) pk[ii] += dot4(f4(Vk + cofs(s, ii)), acc);
      if (k > 0) {
#pragma unroll
        for (int d = 0; d < 4; ++d) pm[d] += dot4(vm[d], acc);
      }
    }
    // sums over the lanes of one column (lane & 3 fixed), then per warp
#pragma unroll
    for (int o = 4; o < 32; o <<= 1) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        pk[q] += __shfl_xor_sync(0xffffffffu, pk[q], o);
        pm[q] += __shfl_xor_sync(0xffffffffu, pm[q], o);
      }
    }
    if (lane < 4) {
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        Pw[warp * 32 + q * 4 + lane] = pk[q];
        Pw[warp * 32 + 16 + q * 4 + lane] = pm[q];
      }
    }
    __syncthreads();
    // ---- classical Gram-Schmidt (pass 0 yields A_k); the last step needs
    // only A_k; between full passes only V_{k-1} and V_k are projected out
    const int passes = (k == r - 1) ? 1 : a.reorth_passes;
    float g[4] = {0.f, 0.f, 0.f, 0.f};                 // Gram row c of the final W
    const int c4 = tid & 3;                            // column of every item of this thread
    for (int pass = 0; pass < passes; ++pass) {
      const bool full = a.reorth_every <= 1 || (k % a.reorth_every) == a.reorth_every - 1;
      const int b0 = (k == r - 1) ? k : (full ? 0 : (k > 0 ? k - 1 : 0));
      const int nb = k + 1 - b0;
      auto blk = [&](int b) -> const float* {
        return b == k ? Vk : (b == k - 1 ? Vkm1 : Vg + (size_t)b * VB);
      };
      // blocks from fl on were projected in the sweep (first pass only)
      const int fl = pass == 0 ? (b0 > k - 1 ? b0 : k - 1) : k + 1;
      const int nbl = fl - b0;                         // blocks projected here
      const int nseg = nbl >= KW ? 1 : (nbl > 0 ? KW / nbl : 1);
      const int items = nbl * nseg;
      for (int w = warp; w < items; w += KW) {
        const int b = b0 + w / nseg, seg = w % nseg;
        const int slo = (nc * seg) / nseg, shi = (nc * (seg + 1)) / nseg;
        const float* Vb = blk(b);
        float acc[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) acc[q] = 0.f;
        for (int s = slo + lane; s < shi; s += 32) {
          float4 v[4], x[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) { v[q] = f4(Vb + cofs(s, q)); x[q] = f4(W + cofs(s, q)); }
#pragma unroll
          for (int ii = 0; ii < 4; ++ii)
#pragma unroll
            for (int c = 0; c < 4; ++c) acc[ii * 4 + c] += dot4(v[ii], x[c]);
        }
        const float tot = tbk::warp_reduce16(acc, lane);
        if ((lane & 1) == 0) Cp[w * 16 + (lane >> 1)] = tot;
      }
      if (nbl > 0) __syncthreads();
      // coefficients of block b, stored by column: Cc[b][c][ii] = (V_b^T W)[ii][c]
      for (int t = tid; t < nb * 16; t += KT) {
        const int bl = t >> 4, q = t & 15, b = b0 + bl;
        float sum = 0.f;
        if (b >= fl) {
          const int h = b == k ? 0 : 16;
#pragma unroll
          for (int w = 0; w < KW; ++w) sum += Pw[w * 32 + h + q];
        } else {
          for (int sg = 0; sg < nseg; ++sg) sum += Cp[(bl * nseg + sg) * 16 + q];
        }
        Cc[b * 16 + (q & 3) * 4 + (q >> 2)] = sum;
      }
      __syncthreads();
      if (pass == 0 && tid < 16) {                     // A_k = V_k^T H V_k, symmetrised
        const int ii = tid >> 2, c = tid & 3;
        tc_block(Ti, 2 * k)[tid] =
            0.5 * ((double)Cc[k * 16 + c * 4 + ii] + (double)Cc[k * 16 + ii * 4 + c]);
      }
      if (k == r - 1) break;
      const bool last = pass == passes - 1;
      // W -= sum_b V_b C_b; on the last pass the Gram matrix of the result.
      // Up to four items per thread at a time, so that the loads of a block
      // (from L2 for the older blocks of a full pass) are in flight together.
      for (int base0 = warp * 32; base0 < D4; base0 += 4 * KT) {
        float4 x[4];
        int sl[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) {
          const int it = base0 + u * KT + lane;
          sl[u] = it < D4 ? it >> 2 : 0;
          x[u] = it < D4 ? f4(W + cofs(sl[u], c4)) : make_float4(0.f, 0.f, 0.f, 0.f);
        }
        for (int b = b0; b <= k; ++b) {
          const float* Vb = blk(b);
          const float4 cf = f4(Cc + b * 16 + 4 * c4);
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (base0 + u * KT >= D4) break;           // uniform over the warp
            x[u] = axpy4(-cf.x, f4(Vb + cofs(sl[u], 0)), x[u]);
            x[u] = axpy4(-cf.y, f4(Vb + cofs(sl[u], 1)), x[u]);
            x[u] = axpy4(-cf.z, f4(Vb + cofs(sl[u], 2)), x[u]);
            x[u] = axpy4(-cf.w, f4(Vb + cofs(sl[u], 3)), x[u]);
          }
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (base0 + u * KT + lane < D4) sf4(W + cofs(sl[u], c4), x[u]);
        if (last) {
          __syncwarp();
#pragma unroll
          for (int u = 0; u < 4; ++u) {
            if (base0 + u * KT + lane >= D4) continue;
#pragma unroll
            for (int e = 0; e < 4; ++e) {                // constant indices into g
              if (e == c4) g[e] += dot4(x[u], x[u]);
              else if (e > c4) g[e] += dot4(x[u], f4(W + cofs(sl[u], e)));
            }
          }
        }
      }
      if (!last) __syncthreads();
    }
    if (k == r - 1) break;
    // ---- in-block QR: W = V_{k+1} B_k
    // chol_state: 0 Cholesky accepted, 1 first factor refused (W untouched),
    // 2 second factor refused (the first one applied)
    int chol_state = 0;
    bool single = false;
    float* src = W;
    float* dst = Vkm1;                                 // free after the projections
    for (int cq = 0; cq < 2; ++cq) {
      float gv[16];
      const int c = tid & 3;
#pragma unroll
      for (int q = 0; q < 16; ++q) gv[q] = ((q >> 2) == c && (q & 3) >= c) ? g[q & 3] : 0.f;
      const float tot = tbk::warp_reduce16(gv, lane);
      if ((lane & 1) == 0) red[warp * 16 + (lane >> 1)] = tot;
      __syncthreads();
      if (warp == 0) {                                 // uniform over the warp
        float G[16], R[16], Ri[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) {
          float sum = 0.f;
#pragma unroll
          for (int w = 0; w < KW; ++w) sum += red[w * 16 + q];
          G[q] = sum;
        }
#pragma unroll
        for (int cc = 0; cc < 4; ++cc)
#pragma unroll
          for (int e = 0; e < cc; ++e) G[cc * 4 + e] = G[e * 4 + cc];
        bool well;
        float dinv[4];
        const bool ok = chol4(G, R, chol_rel, cq == 0 ? chol_abs : 0.0, well, dinv);
        triinv4(R, dinv, Ri);
        if (lane == 0) {
#pragma unroll
          for (int q = 0; q < 16; ++q) { Rsh[q] = R[q]; Rish[q] = Ri[q]; }
          flags[FL_OK] = (ok ? 1 : 0) | (well ? 2 : 0);
          if (cq == 0) {
#pragma unroll
            for (int q = 0; q < 16; ++q) R1s[q] = (double)R[q];
          }
        }
        __syncwarp();
        if (ok && (cq == 1 || well)) {
          // this factor completes the QR: B_k = R (one factor) or R2 R1, one
          // entry per lane, published with T and the column mask by the
          // barrier that ends the step
          if (lane < 16) {
            const int j = lane >> 2, cc = lane & 3;
            double t;
            if (cq == 0) {
              t = (double)Rsh[lane];
            } else {
              t = 0.0;
#pragma unroll
              for (int m = 0; m < 4; ++m) t += (double)Rsh[j * 4 + m] * R1s[m * 4 + cc];
            }
            Bs[lane] = t;
            Bp[lane] = (float)t;
            tc_block(Ti, 2 * k + 1)[lane] = t;
            if (j == cc && !isfinite(t)) tbk::set_status(a.st, TB_ERR_NONFINITE, i);
          }
          if (lane == 0) {
            unsigned long long mask = ((unsigned long long)(unsigned)flags[FL_MASK + 1] << 32) |
                                      (unsigned)flags[FL_MASK];
            mask |= 0xFull << (4 * (k + 1));
            flags[FL_MASK] = (int)(mask & 0xffffffffull);
            flags[FL_MASK + 1] = (int)(mask >> 32);
          }
        }
      }
      __syncthreads();
      const int fl = flags[FL_OK];
      if (!(fl & 1)) { chol_state = cq + 1; break; }
      single = cq == 0 && (fl & 2);
      const bool fin = single || cq == 1;
      // column c of R^-1 (upper triangular: rows j <= c)
      const float ric[4] = {Rish[c], Rish[4 + c], Rish[8 + c], Rish[12 + c]};
#pragma unroll
      for (int q = 0; q < 4; ++q) g[q] = 0.f;
      float* const out = cq == 0 ? dst : W;
      for (int base = warp * 32; base < D4; base += KT) {
        const int it = base + lane;
        const bool on = it < D4;
        const int s = on ? it >> 2 : 0;
        const float* xs = cq == 0 ? src : dst;
        float4 y = make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
        for (int j = 0; j < 4; ++j)
          if (j <= c) y = axpy4(ric[j], f4(xs + cofs(s, j)), y);
        __syncwarp();                                  // every lane has read its slot
        if (on) {
          sf4(out + cofs(s, c), y);
          if (fin) {
            sf4(Vg + (size_t)(k + 1) * VB + cofs(s, c), y);
            if constexpr (BF) vbf[SPB * s + c] = pack_bf16x4(y);
          }
        }
        if (!fin) {                                    // Gram matrix for the second factor
          __syncwarp();
          if (on) {
#pragma unroll
            for (int e = 0; e < 4; ++e) {
              if (e == c) g[e] += dot4(y, y);
              else if (e > c) g[e] += dot4(y, f4(out + cofs(s, e)));
            }
          }
        }
      }
      if (fin) break;
    }
    // V_{k+1} is in dst after one factor (or MGS on W), in W after two
    float* Vn = (chol_state == 1 || (chol_state == 0 && single)) ? dst : W;
    int act = 0xF;
    if (chol_state != 0) {
      // modified Gram-Schmidt by warp 0 on the columns of the last written
      // block, a column dropped when its norm is <= defl_tol
      float* S = chol_state == 1 ? W : dst;
      float* O = chol_state == 1 ? dst : W;
      __syncthreads();
      if (warp == 0) {
        double* const R = Rm;                          // written by lane 0 only
        if (lane == 0) {
#pragma unroll
          for (int q = 0; q < 16; ++q) R[q] = 0.0;
        }
        int mact = 0;
        bool nonfinite = false;
        auto at = [](int row, int col) { return cofs(row >> 2, col) + (row & 3); };
        for (int c = 0; c < 4; ++c) {
          for (int ps = 0; ps < 2 && c > 0; ++ps) {
            float dd[3] = {0.f, 0.f, 0.f};
            for (int row = lane; row < D4; row += 32) {
              const float w = S[at(row, c)];
#pragma unroll
              for (int j = 0; j < 3; ++j) if (j < c) dd[j] += O[at(row, j)] * w;
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) if (j < c) dd[j] = tbk::warp_sum(dd[j]);
            for (int row = lane; row < D4; row += 32) {
              float w = S[at(row, c)];
#pragma unroll
              for (int j = 0; j < 3; ++j) if (j < c) w -= dd[j] * O[at(row, j)];
              S[at(row, c)] = w;
            }
            if (lane == 0) {
#pragma unroll
              for (int j = 0; j < 3; ++j) if (j < c) R[j * 4 + c] += (double)dd[j];
            }
          }
          float nn = 0.f;
          for (int row = lane; row < D4; row += 32) {
            const float w = S[at(row, c)];
            nn += w * w;
          }
          nn = tbk::warp_sum(nn);
          const double nrm = sqrt((double)nn);
          if (!isfinite(nrm)) nonfinite = true;
          const bool keep = nrm > a.defl_tol;
          const float inv = keep ? (float)(1.0 / nrm) : 0.f;
          for (int row = lane; row < D4; row += 32) O[at(row, c)] = S[at(row, c)] * inv;
          if (keep) {
            if (lane == 0) R[c * 4 + c] = nrm;
            mact |= 1 << c;
          }
          __syncwarp();
        }
        // copies of V_{k+1}: the basis slot and (BF16) the sweep's copy
        for (int q = lane; q < SP * nc; q += 32) Vg[(size_t)(k + 1) * VB + q] = O[q];
        if constexpr (BF) {
          for (int q = lane; q < 4 * nc; q += 32)
            vbf[SPB * (q >> 2) + (q & 3)] = pack_bf16x4(f4(O + cofs(q >> 2, q & 3)));
        }
        if (lane == 0) {
          if (chol_state == 2) {                       // S was W R1^-1: B_k = R_mgs R1
#pragma unroll
            for (int rr = 0; rr < 4; ++rr)
#pragma unroll
              for (int c = 0; c < 4; ++c) {
                double t = 0.0;
#pragma unroll
                for (int j = 0; j < 4; ++j) t += R[rr * 4 + j] * R1s[j * 4 + c];
                Bs[rr * 4 + c] = t;
              }
          } else {
#pragma unroll
            for (int q = 0; q < 16; ++q) Bs[q] = R[q];
          }
          flags[FL_ACT] = mact;
          if (nonfinite) tbk::set_status(a.st, TB_ERR_NONFINITE, i);
        }
      }
      Vn = O;
      __syncthreads();
      act = flags[FL_ACT];
      if (tid < 16) {
        tc_block(Ti, 2 * k + 1)[tid] = Bs[tid];
        Bp[tid] = (float)Bs[tid];
      }
      if (tid == 0) {
        unsigned long long mask = ((unsigned long long)(unsigned)flags[FL_MASK + 1] << 32) |
                                  (unsigned)flags[FL_MASK];
        mask |= (unsigned long long)act << (4 * (k + 1));
        flags[FL_MASK] = (int)(mask & 0xffffffffull);
        flags[FL_MASK + 1] = (int)(mask >> 32);
        if (!isfinite(Bs[0] + Bs[5] + Bs[10] + Bs[15])) tbk::set_status(a.st, TB_ERR_NONFINITE, i);
      }
    }
    __syncthreads();                                   // V_{k+1}, B_k and the mask complete
    // rotate: V_{k+1} becomes V_k, V_k becomes V_{k-1}, the third buffer W
    {
      float* o0 = Vk;
      float* o1 = Vkm1;
      float* o2 = W;
      Vkm1 = o0;
      Vk = Vn;
      W = (Vn == o1) ? o2 : o1;
    }
    if (act == 0) break;
    nblocks = k + 2;
  }
  // ---- outputs: column mask, rows of V for the target and its H neighbours
  if (tid == 0)
    a.colmask[i] = ((unsigned long long)(unsigned)flags[FL_MASK + 1] << 32) | (unsigned)flags[FL_MASK];
  {
    const size_t ybase = (size_t)(i + a.h_off[i]) * 4;
    const int nrows = (deg + 1) * 4;
    const int rcnt = roff[1] - roff[0];
    for (int q = tid; q < nrows * NT; q += KT) {
      const int rr = q / NT, col = q - rr * NT;
      const int qq = rr >> 2, beta = rr & 3;
      const int e = roff[0] + qq - 1;       // entry of neighbour qq - 1 in row 0
      const int so = qq == 0 ? 0 : (qq - 1 < rcnt ? (ovf ? bref[e].y : rsl[e]) : -1);
      const int b = col >> 2, c = col & 3;
      float val = 0.f;
      if (b < nblocks && so >= 0) val = Vg[(size_t)b * VB + (so ^ (4 * c)) + beta];
      a.Y[(ybase + rr) * NT + col] = val;
    }
  }
  __syncthreads();
}

}  // namespace tbsk
