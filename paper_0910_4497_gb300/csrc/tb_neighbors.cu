// a1: neighbour and cluster lists (Sec. 2: atoms within the cutoff radius).
//
// Brute force over all pairs, tiled through shared memory: a CTA of 8 warps
// serves 8 target atoms and streams the candidate positions once per tile.
// An FP32 minimum-image distance with a 0.01 A margin prefilters candidates;
// membership is decided by the FP64 test (each operation separately rounded,
// no FMA), which makes the lists bit-exact:
//   d = x_j - x_i;  d -= L if d > L/2;  d += L if d < -L/2;
//   r2 = (dx*dx + dy*dy) + dz*dz <= R*R.
// Lists are compacted with warp ballots, so they come out in ascending j.
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

}  // namespace

tb_status launch_neighbors(tb_ctx* c, int n, const double* pos, double L, int* h_off,
                           int* h_idx, int* c_off, int* c_idx, cudaStream_t s) {
  const tb_params& p = c->p;
  float4* posf = reinterpret_cast<float4*>(c->rho);   // scratch: rho is free here
  pos_to_f32_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, pos, L, posf, c->d_status);
  const double R2h = p.rm * p.rm, R2c = p.Rc * p.Rc;
  const float Rh_pre2 = (float)((p.rm + 0.01) * (p.rm + 0.01));
  const float Rc_pre2 = (float)((p.Rc + 0.01) * (p.Rc + 0.01));
  const int grid = (n + NB_WARPS - 1) / NB_WARPS;
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
