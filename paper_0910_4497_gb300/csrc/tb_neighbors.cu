// Neighbour and cluster lists (Sec. 2: atoms within the cutoff radius).
//
// Brute force over all pairs, tiled through shared memory: a CTA of 8 warps
// serves 8 target atoms and streams the candidate positions once per tile.
// An FP32 minimum-image distance with a 0.01 A margin prefilters candidates;
// membership is decided by the FP64 test (each operation separately rounded,
// no FMA), which makes the lists bit-exact:
//   d = x_j - x_i;  d -= L if d > L/2;  d += L if d < -L/2;
//   r2 = (dx*dx + dy*dy) + dz*dz <= R*R.
// Lists are compacted with warp ballots, so they come out in ascending j.
//
// When the box holds at least three cells of side >= Rc + 0.01 A per
// dimension, the candidates come from cell lists instead: atoms are binned
// (counting sort), a warp per target scans the 27 surrounding cells with the
// same two-stage test, sorts what it found (bitonic, in shared memory) and
// writes padded per-atom lists that are then compacted into the CSR.  The
// 0.01 A margin keeps every pair within Rc in adjacent cells whatever the
// rounding of the cell assignment.
#include "tb_internal.cuh"

namespace {

constexpr int NB_WARPS = 8;
constexpr int NB_THREADS = NB_WARPS * 32;

__global__ void pos_to_f32_kernel(int n, const double* __restrict__ pos, double L,
                                  float4* __restrict__ posf, int* st) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  bool ok = (x >= 0.0 && x < L) && (y >= 0.0 && y < L) && (z >= 0.0 && z < L);
  if (!ok) tbk::set_status(st, TB_ERR_INVALID_ARG, i);
  posf[i] = make_float4((float)x, (float)y, (float)z, 0.f);
}

// Nearest periodic image of a separation d in (-L, L).
__device__ __forceinline__ double min_image_rn(double d, double L, double h) {
  return d > h ? __dsub_rn(d, L) : (d < -h ? __dadd_rn(d, L) : d);
}

// MODE 0: count (writes hcnt/ccnt); MODE 1: fill the CSR lists.
template <int MODE>
__global__ void __launch_bounds__(NB_THREADS)
nbr_kernel(int n, const double* __restrict__ pos, const float4* __restrict__ posf,
           double L, double R2h, double R2c, float Rh_pre2, float Rc_pre2,
           int* __restrict__ hcnt, int* __restrict__ ccnt,
           const int* __restrict__ h_off, int* __restrict__ h_idx,
           const int* __restrict__ c_off, int* __restrict__ c_idx,
           int max_h, int max_c, int* st) {
  __shared__ float4 tile[NB_THREADS];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int i = blockIdx.x * NB_WARPS + warp;
  const bool active = i < n;
  const float Lf = (float)L, invLf = (float)(1.0 / L);
  float4 pi = active ? posf[i] : make_float4(0.f, 0.f, 0.f, 0.f);
  double xi = 0, yi = 0, zi = 0;
  if (active) { xi = pos[3 * i]; yi = pos[3 * i + 1]; zi = pos[3 * i + 2]; }
  int nh = 0, ncl = 1;  // cluster slot 0 is the target itself
  int hbase = 0, cbase = 0;
  if (MODE == 1 && active) {
    hbase = h_off[i];
    cbase = c_off[i];
    if (lane == 0 && max_c > 0) c_idx[cbase] = i;
  }
  for (int t0 = 0; t0 < n; t0 += NB_THREADS) {
    __syncthreads();
    int jt = t0 + threadIdx.x;
    tile[threadIdx.x] = jt < n ? posf[jt] : make_float4(0.f, 0.f, 0.f, 0.f);
    __syncthreads();
    if (!active) continue;
    const int tn = min(NB_THREADS, n - t0);
    for (int c = 0; c < tn; c += 32) {
      const int jl = c + lane;
      const int j = t0 + jl;
      bool in_h = false, in_c = false;
      if (jl < tn && j != i) {
        float4 pj = tile[jl];
        float dx = pj.x - pi.x, dy = pj.y - pi.y, dz = pj.z - pi.z;
        dx -= Lf * rintf(dx * invLf);
        dy -= Lf * rintf(dy * invLf);
        dz -= Lf * rintf(dz * invLf);
        float r2f = dx * dx + dy * dy + dz * dz;
        if (r2f <= Rc_pre2 || r2f <= Rh_pre2) {
          const double hL = 0.5 * L;
          double ex = min_image_rn(__dsub_rn(pos[3 * j], xi), L, hL);
          double ey = min_image_rn(__dsub_rn(pos[3 * j + 1], yi), L, hL);
          double ez = min_image_rn(__dsub_rn(pos[3 * j + 2], zi), L, hL);
          double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)),
                                __dmul_rn(ez, ez));
          in_h = r2 <= R2h;
          in_c = r2 <= R2c;
        }
      }
      unsigned bh = __ballot_sync(0xffffffffu, in_h);
      unsigned bc = __ballot_sync(0xffffffffu, in_c);
      if (MODE == 1) {
        unsigned below = (1u << lane) - 1u;
        int ph = nh + __popc(bh & below);
        int pc = ncl + __popc(bc & below);
        if (in_h && ph < max_h) h_idx[hbase + ph] = j;
        if (in_c && pc < max_c) c_idx[cbase + pc] = j;
      }
      nh += __popc(bh);
      ncl += __popc(bc);
    }
  }
  if (MODE == 0 && active && lane == 0) {
    if (nh > max_h) tbk::set_status(st, TB_ERR_CAPACITY, nh);
    if (ncl > max_c) tbk::set_status(st, TB_ERR_CAPACITY, ncl);
    hcnt[i] = min(nh, max_h);
    ccnt[i] = min(ncl, max_c);
  }
}

// Exclusive scans of two count arrays (length n) into CSR offsets (length n+1).
__global__ void __launch_bounds__(1024)
scan2_kernel(int n, const int* __restrict__ a, int* __restrict__ oa,
             const int* __restrict__ b, int* __restrict__ ob) {
  __shared__ int sa[1024], sb[1024];
  const int t = threadIdx.x;
  const int chunk = (n + 1023) / 1024;
  const int lo = min(n, t * chunk), hi = min(n, lo + chunk);
  int s1 = 0, s2 = 0;
  for (int k = lo; k < hi; ++k) { s1 += a[k]; s2 += b[k]; }
  sa[t] = s1;
  sb[t] = s2;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    int v1 = t >= o ? sa[t - o] : 0, v2 = t >= o ? sb[t - o] : 0;
    __syncthreads();
    sa[t] += v1;
    sb[t] += v2;
    __syncthreads();
  }
  int r1 = sa[t] - s1, r2 = sb[t] - s2;
  for (int k = lo; k < hi; ++k) {
    oa[k] = r1; ob[k] = r2;
    r1 += a[k]; r2 += b[k];
  }
  if (t == 1023) { oa[n] = sa[1023]; ob[n] = sb[1023]; }
}

// ---------------------------------------------------------------- cell lists

__device__ __forceinline__ int cell_coord(double x, double L, int nc) {
  int c = (int)(x * (double)nc / L);
  return c < 0 ? 0 : (c >= nc ? nc - 1 : c);
}

// The FP32 copy of the positions and its [0, L) check (as pos_to_f32_kernel),
// then each atom's cell and the cells' counts.
__global__ void cell_assign_kernel(int n, const double* __restrict__ pos, double L, int nc,
                                   float4* __restrict__ posf, int* st,
                                   int* __restrict__ atom_cell, int* __restrict__ cell_cnt) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const double x = pos[3 * i], y = pos[3 * i + 1], z = pos[3 * i + 2];
  const bool ok = (x >= 0.0 && x < L) && (y >= 0.0 && y < L) && (z >= 0.0 && z < L);
  if (!ok) tbk::set_status(st, TB_ERR_INVALID_ARG, i);
  posf[i] = make_float4((float)x, (float)y, (float)z, 0.f);
  const int cx = cell_coord(x, L, nc), cy = cell_coord(y, L, nc), cz = cell_coord(z, L, nc);
  const int c = (cx * nc + cy) * nc + cz;
  atom_cell[i] = c;
  atomicAdd(&cell_cnt[c], 1);
}

__global__ void cell_fill_kernel(int n, const int* __restrict__ atom_cell,
                                 const int* __restrict__ cell_off, int* __restrict__ cell_fill,
                                 int* __restrict__ cell_atoms) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  const int c = atom_cell[i];
  cell_atoms[cell_off[c] + atomicAdd(&cell_fill[c], 1)] = i;
}

// Exclusive scan of one count array (length m) into offsets (length m+1); the
// counts are zeroed as they are read (they serve next as the fill cursors).
__global__ void __launch_bounds__(1024) scan1_kernel(int m, int* __restrict__ a,
                                                     int* __restrict__ oa) {
  __shared__ int sa[1024];
  const int t = threadIdx.x;
  const int chunk = (m + 1023) / 1024;
  const int lo = min(m, t * chunk), hi = min(m, lo + chunk);
  int s1 = 0;
  for (int k = lo; k < hi; ++k) s1 += a[k];
  sa[t] = s1;
  __syncthreads();
  for (int o = 1; o < 1024; o <<= 1) {
    const int v1 = t >= o ? sa[t - o] : 0;
    __syncthreads();
    sa[t] += v1;
    __syncthreads();
  }
  int r1 = sa[t] - s1;
  for (int k = lo; k < hi; ++k) {
    oa[k] = r1;
    r1 += a[k];
    a[k] = 0;
  }
  if (t == 1023) oa[m] = sa[1023];
}

// Ascending bitonic sort of v[0..len) (len a power of two) by one warp.
__device__ __forceinline__ void warp_bitonic(int* v, int len, int lane) {
  for (int k = 2; k <= len; k <<= 1)
    for (int j = k >> 1; j > 0; j >>= 1) {
      for (int x = lane; x < len; x += 32) {
        const int y = x ^ j;
        if (y > x) {
          const int a = v[x], b = v[y];
          const bool up = (x & k) == 0;
          if ((a > b) == up) { v[x] = b; v[y] = a; }
        }
      }
      __syncwarp();
    }
}

// One warp per target: candidates from the 27 cells around the target's cell,
// the same FP32 prefilter and FP64 membership test as nbr_kernel, then sorted
// lists written into padded per-atom rows (counts capped at the capacities).
// The candidates that pass the prefilter are staged in shared memory and the
// FP64 test runs on the compacted list: a warp-wide FP64 instruction costs
// the same with one active lane as with 32, and most 32-atom batches of the
// cells hold only a few atoms near the target.
__global__ void __launch_bounds__(NB_THREADS)
nbr_cell_kernel(int n, const double* __restrict__ pos, const float4* __restrict__ posf,
                double L, double R2h, double R2c, float Rh_pre2, float Rc_pre2, int nc,
                const int* __restrict__ atom_cell, const int* __restrict__ cell_off,
                const int* __restrict__ cell_atoms, int capc, int caph, int* __restrict__ hcnt,
                int* __restrict__ ccnt, int* __restrict__ pad_h, int* __restrict__ pad_c,
                int max_h, int max_c, int* st) {
  extern __shared__ int nb_smem[];
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  int* cand_c = nb_smem + warp * (2 * capc + caph + 64);
  int* cand_h = cand_c + capc;                         // caph Hamiltonian neighbours
  int* stg = cand_h + caph;                            // capc staged candidates
  int* cex = stg + capc;                               // 32: start of each cell's candidates
  int* cbg = cex + 32;                                 // 32: its first index in cell_atoms
  const int i = blockIdx.x * NB_WARPS + warp;
  if (i >= n) return;
  const float Lf = (float)L, invLf = (float)(1.0 / L);
  const float4 pi = posf[i];
  const double xi = pos[3 * i], yi = pos[3 * i + 1], zi = pos[3 * i + 2];
  const double hL = 0.5 * L;
  const int ci = atom_cell[i];
  const int cx = ci / (nc * nc), cy = (ci / nc) % nc, cz = ci % nc;
  int nh = 0, ncand = 0, nstg = 0;
  const unsigned below = (1u << lane) - 1u;
  // FP64 membership test of the staged candidates, 32 at a time
  auto flush = [&]() {
    __syncwarp();
    for (int b = 0; b < nstg; b += 32) {
      const int x = b + lane;
      bool in_h = false, in_c = false;
      int j = -1;
      if (x < nstg) {
        j = stg[x];
        const double ex = min_image_rn(__dsub_rn(pos[3 * j], xi), L, hL);
        const double ey = min_image_rn(__dsub_rn(pos[3 * j + 1], yi), L, hL);
        const double ez = min_image_rn(__dsub_rn(pos[3 * j + 2], zi), L, hL);
        const double r2 = __dadd_rn(__dadd_rn(__dmul_rn(ex, ex), __dmul_rn(ey, ey)),
                                    __dmul_rn(ez, ez));
        in_h = r2 <= R2h;
        in_c = r2 <= R2c;
      }
      const unsigned bh = __ballot_sync(0xffffffffu, in_h);
      const unsigned bc = __ballot_sync(0xffffffffu, in_c);
      const int ph = nh + __popc(bh & below), pc = ncand + __popc(bc & below);
      if (in_h && ph < caph) cand_h[ph] = j;
      if (in_c && pc < capc) cand_c[pc] = j;
      nh += __popc(bh);
      ncand += __popc(bc);
    }
    __syncwarp();
    nstg = 0;
  };
  // the 27 cells' ranges in one round of loads (lane q: cell q), their
  // candidates numbered by an exclusive scan; each lane finds the cell of its
  // candidate by binary search
  {
    int cb = 0, cn = 0;
    if (lane < 27) {
      const int ox = lane / 9 - 1, oy = (lane / 3) % 3 - 1, oz = lane % 3 - 1;
      const int c2 = (((cx + ox + nc) % nc) * nc + (cy + oy + nc) % nc) * nc + (cz + oz + nc) % nc;
      cb = cell_off[c2];
      cn = cell_off[c2 + 1] - cb;
    }
    int incl = cn;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    cex[lane] = incl - cn;
    cbg[lane] = cb;
    const int total = __shfl_sync(0xffffffffu, incl, 31);
    __syncwarp();
    // candidate x: its cell (the last q with cex[q] <= x) and atom index
    auto cand_atom = [&](int x) -> int {
      if (x >= total) return -1;
      int lo = 0, hi = 26;
      while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (cex[mid] <= x) lo = mid; else hi = mid - 1;
      }
      return cell_atoms[cbg[lo] + (x - cex[lo])];
    };
    // four batches of 32 per round: the four atom-index loads in flight, then
    // the four position loads, then the FP32 prefilter; staged in batch order
    for (int b = 0; b < total; b += 128) {
      int j[4];
      float4 pj[4];
#pragma unroll
      for (int u = 0; u < 4; ++u) j[u] = cand_atom(b + 32 * u + lane);
#pragma unroll
      for (int u = 0; u < 4; ++u) pj[u] = j[u] >= 0 ? posf[j[u]] : make_float4(0.f, 0.f, 0.f, 0.f);
#pragma unroll
      for (int u = 0; u < 4; ++u) {
        bool pass = false;
        if (j[u] >= 0 && j[u] != i) {
          float dx = pj[u].x - pi.x, dy = pj[u].y - pi.y, dz = pj[u].z - pi.z;
          dx -= Lf * rintf(dx * invLf);
          dy -= Lf * rintf(dy * invLf);
          dz -= Lf * rintf(dz * invLf);
          const float r2f = dx * dx + dy * dy + dz * dz;
          pass = r2f <= Rc_pre2 || r2f <= Rh_pre2;
        }
        const unsigned bp = __ballot_sync(0xffffffffu, pass);
        if (nstg + __popc(bp) > capc) flush();          // keep the stage within capacity
        if (pass) stg[nstg + __popc(bp & below)] = j[u];
        nstg += __popc(bp);
      }
    }
  }
  flush();
  // pad to a power of two with INT_MAX, sort ascending
  const int kc = min(ncand, capc), kh = min(nh, caph);
  int lc = 1;
  while (lc < kc) lc <<= 1;
  int lh = 1;
  while (lh < kh) lh <<= 1;
  for (int x = kc + lane; x < lc; x += 32) cand_c[x] = 0x7fffffff;
  for (int x = kh + lane; x < lh; x += 32) cand_h[x] = 0x7fffffff;
  __syncwarp();
  warp_bitonic(cand_c, lc, lane);
  warp_bitonic(cand_h, lh, lane);
  const int wc = min(ncand + 1, max_c), wh = min(nh, max_h);
  int* rc = pad_c + (size_t)i * max_c;
  int* rh = pad_h + (size_t)i * max_h;
  if (lane == 0 && max_c > 0) rc[0] = i;
  for (int x = lane; x + 1 < wc; x += 32) rc[x + 1] = cand_c[x];
  for (int x = lane; x < wh; x += 32) rh[x] = cand_h[x];
  if (lane == 0) {
    if (nh > max_h) tbk::set_status(st, TB_ERR_CAPACITY, nh);
    if (ncand + 1 > max_c) tbk::set_status(st, TB_ERR_CAPACITY, ncand + 1);
    hcnt[i] = wh;
    ccnt[i] = wc;
  }
}

// Padded per-atom rows -> CSR (one warp per atom).
__global__ void __launch_bounds__(NB_THREADS)
compact_kernel(int n, const int* __restrict__ pad_h, const int* __restrict__ pad_c, int max_h,
               int max_c, const int* __restrict__ h_off, int* __restrict__ h_idx,
               const int* __restrict__ c_off, int* __restrict__ c_idx) {
  const int lane = threadIdx.x & 31;
  const int i = blockIdx.x * NB_WARPS + (threadIdx.x >> 5);
  if (i >= n) return;
  const int h0 = h_off[i], hn = h_off[i + 1] - h0;
  const int c0 = c_off[i], cn = c_off[i + 1] - c0;
  for (int x = lane; x < hn; x += 32) h_idx[h0 + x] = pad_h[(size_t)i * max_h + x];
  for (int x = lane; x < cn; x += 32) c_idx[c0 + x] = pad_c[(size_t)i * max_c + x];
}

}  // namespace

size_t neighbor_cell_capacity(int n) { return (size_t)(n < 32 ? 64 : 2 * n); }

// Kernels launch_neighbors issues for a box of side L (the same path choice).
int neighbor_kernel_count(const tb_ctx* c, double L) {
  const tb_params& p = c->p;
  int nc = (int)(L / (p.Rc + 0.01));
  while (nc >= 3 && (size_t)nc * nc * nc > neighbor_cell_capacity(c->reserved_n)) --nc;
  return (nc >= 3 && p.max_cluster <= 512) ? 6 : 4;
}

tb_status launch_neighbors(tb_ctx* c, int n, const double* pos, double L, int* h_off,
                           int* h_idx, int* c_off, int* c_idx, cudaStream_t s) {
  const tb_params& p = c->p;
  float4* posf = reinterpret_cast<float4*>(c->rho);   // scratch: rho is free here
  const double R2h = p.rm * p.rm, R2c = p.Rc * p.Rc;
  const float Rh_pre2 = (float)((p.rm + 0.01) * (p.rm + 0.01));
  const float Rc_pre2 = (float)((p.Rc + 0.01) * (p.Rc + 0.01));
  const int grid = (n + NB_WARPS - 1) / NB_WARPS;
  // cells of side >= Rc + 0.01 A, at least 3 per dimension, at most the capacity
  int nc = (int)(L / (p.Rc + 0.01));
  while (nc >= 3 && (size_t)nc * nc * nc > neighbor_cell_capacity(c->reserved_n)) --nc;
  const int capc = p.max_cluster <= 128 ? 128 : (p.max_cluster <= 256 ? 256 : 512);
  const int caph = p.max_hnbr <= 64 ? 64 : (p.max_hnbr <= 128 ? 128 : 256);
  const size_t cell_smem = (size_t)NB_WARPS * (2 * capc + caph + 64) * sizeof(int);
  if (nc >= 3 && p.max_cluster <= 512) {
    const int ncell = nc * nc * nc;
    TB_CUDA_TRY(cudaMemsetAsync(c->cell_cnt, 0, sizeof(int) * ncell, s));
    cell_assign_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, pos, L, nc, posf, c->d_status,
                                                       c->atom_cell, c->cell_cnt);
    scan1_kernel<<<1, 1024, 0, s>>>(ncell, c->cell_cnt, c->cell_off);   // counts back to zero
    cell_fill_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, c->atom_cell, c->cell_off, c->cell_cnt,
                                                     c->cell_atoms);
    nbr_cell_kernel<<<grid, NB_THREADS, cell_smem, s>>>(
        n, pos, posf, L, R2h, R2c, Rh_pre2, Rc_pre2, nc, c->atom_cell, c->cell_off,
        c->cell_atoms, capc, caph, c->scan_h, c->scan_c, c->pad_h, c->pad_c, p.max_hnbr,
        p.max_cluster, c->d_status);
    scan2_kernel<<<1, 1024, 0, s>>>(n, c->scan_h, h_off, c->scan_c, c_off);
    compact_kernel<<<grid, NB_THREADS, 0, s>>>(n, c->pad_h, c->pad_c, p.max_hnbr, p.max_cluster,
                                              h_off, h_idx, c_off, c_idx);
    TB_CUDA_TRY(cudaGetLastError());
    return TB_OK;
  }
  pos_to_f32_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, pos, L, posf, c->d_status);
  nbr_kernel<0><<<grid, NB_THREADS, 0, s>>>(n, pos, posf, L, R2h, R2c, Rh_pre2, Rc_pre2,
                                            c->scan_h, c->scan_c, nullptr, nullptr,
                                            nullptr, nullptr, p.max_hnbr,
                                            p.max_cluster, c->d_status);
  scan2_kernel<<<1, 1024, 0, s>>>(n, c->scan_h, h_off, c->scan_c, c_off);
  nbr_kernel<1><<<grid, NB_THREADS, 0, s>>>(n, pos, posf, L, R2h, R2c, Rh_pre2, Rc_pre2,
                                            nullptr, nullptr, h_off, h_idx, c_off,
                                            c_idx, p.max_hnbr, p.max_cluster,
                                            c->d_status);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}
