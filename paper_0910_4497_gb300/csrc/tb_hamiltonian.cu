// Hamiltonian blocks of Eq. (1) for every directed bond i -> j.
//
// Slater-Koster table for s and p orbitals with direction cosines l of
// d = R_j - R_i (minimum image):
//   ss = Vss, s_i p_j(g) = l_g Vsp, p_i(g) s_j = -l_g Vsp,
//   p_i(g) p_j(h) = l_g l_h (Vpps - Vppp) + delta_gh Vppp,
// each times the distance scaling s(r).  The gradient block is
//   dt/dd_k = s'(r) l_k M(l) + s(r) dM/dd_k,  dl_g/dd_k = (delta_gk - l_g l_k)/r.
// One thread per bond; runs of 32 consecutive bonds (one warp) are dealt out
// to the warps of all blocks in turn, so that every SM gets a share of this
// FP64-bound work in full warps whatever the bond count; the source atom is
// found by binary search in h_off.  For the mixed and BF16 paths the bond's
// Slater-Koster record (s(r), l) goes out as one float4: the sweeps rebuild
// the block's action from it (16 bytes per bond instead of a 64-byte block).
#include "tb_internal.cuh"
#include "tb_model.cuh"

namespace {

struct SK {
  double Vss, Vsp, Vpps, Vppp;
};

__global__ void __launch_bounds__(256)
assemble_kernel(int n, const double* __restrict__ pos, double L,
                const int* __restrict__ h_off, const int* __restrict__ h_idx,
                tb_gsp g, SK sk, double* __restrict__ Hblk, double* __restrict__ dHblk,
                float4* __restrict__ Hsk, int* st) {
  const int nb = h_off[n];
  const int wg = blockIdx.x + gridDim.x * (threadIdx.x >> 5);     // warps interleaved over blocks
  const int stride = gridDim.x * blockDim.x;
  for (int pidx = wg * 32 + (threadIdx.x & 31); pidx < nb; pidx += stride) {
  int lo = 0, hi = n;                 // source atom: h_off[i] <= pidx < h_off[i+1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (h_off[mid] <= pidx) lo = mid; else hi = mid;
  }
  const int i = lo;
  const int j = h_idx[pidx];
  const double hL = 0.5 * L;
  double d[3];
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    const double x = pos[3 * j + k] - pos[3 * i + k];
    d[k] = x > hL ? x - L : (x < -hL ? x + L : x);
  }
  const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  if (!(r > 0.0)) {
    tbk::set_status(st, TB_ERR_NONFINITE, i);
    continue;
  }
  double s, ds;
  tb_gsp_eval(g, r, s, ds);
  const double inv = 1.0 / r;
  const double l[3] = {d[0] * inv, d[1] * inv, d[2] * inv};
  const double dpp = sk.Vpps - sk.Vppp;
  double M[16];
  M[0] = sk.Vss;
#pragma unroll
  for (int a = 0; a < 3; ++a) {
    M[1 + a] = l[a] * sk.Vsp;
    M[4 * (1 + a)] = -l[a] * sk.Vsp;
#pragma unroll
    for (int b = 0; b < 3; ++b)
      M[4 * (1 + a) + 1 + b] = l[a] * l[b] * dpp + (a == b ? sk.Vppp : 0.0);
  }
  double* H = Hblk + (size_t)pidx * 16;
#pragma unroll
  for (int q = 0; q < 16; ++q) H[q] = s * M[q];
  if (Hsk) Hsk[pidx] = make_float4((float)s, (float)l[0], (float)l[1], (float)l[2]);
  double* Gd = dHblk + (size_t)pidx * 48;
#pragma unroll
  for (int k = 0; k < 3; ++k) {
    double dl[3];
#pragma unroll
    for (int a = 0; a < 3; ++a) dl[a] = ((a == k ? 1.0 : 0.0) - l[a] * l[k]) * inv;
    double dM[16];
    dM[0] = 0.0;
#pragma unroll
    for (int a = 0; a < 3; ++a) {
      dM[1 + a] = dl[a] * sk.Vsp;
      dM[4 * (1 + a)] = -dl[a] * sk.Vsp;
#pragma unroll
      for (int b = 0; b < 3; ++b)
        dM[4 * (1 + a) + 1 + b] = (dl[a] * l[b] + l[a] * dl[b]) * dpp;
    }
#pragma unroll
    for (int q = 0; q < 16; ++q) Gd[16 * k + q] = ds * l[k] * M[q] + s * dM[q];
  }
  }
}

}  // namespace

tb_status launch_assemble(tb_ctx* c, int n, const double* pos, double L,
                          const int* h_off, const int* h_idx, double* Hblk,
                          double* dHblk, float* Hsk, cudaStream_t s) {
  const tb_params& p = c->p;
  SK sk{p.Vss, p.Vsp, p.Vpps, p.Vppp};
  const int threads = 64;
  const int grid = 16 * c->num_sms;                 // up to 32 warps per SM
  assemble_kernel<<<grid, threads, 0, s>>>(n, pos, L, h_off, h_idx, tb_hopping_gsp(p),
                                           sk, Hblk, dHblk, reinterpret_cast<float4*>(Hsk),
                                           c->d_status);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}
