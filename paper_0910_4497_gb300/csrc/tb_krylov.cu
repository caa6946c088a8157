// a3-a5: per-target cluster map and block Lanczos (Sec. 3, Eq. (Krylov) and
// the block form of Eqs. (lanczos) / (lanczos_blas3)).
//
// One CTA per target atom (persistent, grid-stride over targets).  For target
// i with cluster atoms cl[0..nc) (cl[0] = i, the rest ascending):
//   * the local sparsity of H_c is built in the CTA: for each slot s and each
//     Hamiltonian neighbour of cl[s] that is in the cluster, (local slot,
//     global bond index).  H_c is never formed: its 4x4 blocks are read from
//     the global bond table (FP64, or its FP32 mirror) during each sweep;
//   * V_1 = E_i (the target's four orbitals, slot 0), B_0 = 0, and for
//     k = 1..r:
//       W = H_c V_k - V_{k-1} B_{k-1}^T        (block sparse sweep, 4 columns)
//       A_k = V_k^T W;  W -= V_k A_k
//       passes x: C = Q^T W, W -= Q C           (Q = V_1..V_k, classical GS)
//       W = V_{k+1} B_k                         (in-block MGS, two passes per
//                                                column, column dropped when its
//                                                norm is <= defl_tol)
//     T gets A_k on the diagonal and B_k / B_k^T off the diagonal;
//   * the rows of V belonging to the target and its Hamiltonian neighbours are
//     written out (Y) for the density-matrix columns.
// The basis lives in shared memory when r * 4 * max_cluster * 4 values fit,
// otherwise in a per-CTA slot of global memory (L2-resident).
// Layout of the basis: block b occupies Dmax*4 values, row-major [row][4].
#include "tb_internal.cuh"

namespace {

constexpr int KT = 256;
constexpr int KW = KT / 32;
// flags[0..KW): warp totals of the block scan; then the column mask and the
// active-column bits of the newest block.
constexpr int FL_MASK = KW;
constexpr int FL_ACT = KW + 2;

__device__ __forceinline__ void load_h(const double* __restrict__ H, int blk, double h[16]) {
  const double2* p = reinterpret_cast<const double2*>(H + (size_t)blk * 16);
#pragma unroll
  for (int q = 0; q < 8; ++q) {
    double2 v = __ldg(p + q);
    h[2 * q] = v.x;
    h[2 * q + 1] = v.y;
  }
}
__device__ __forceinline__ void load_h(const float* __restrict__ H, int blk, float h[16]) {
  const float4* p = reinterpret_cast<const float4*>(H + (size_t)blk * 16);
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    float4 v = __ldg(p + q);
    h[4 * q] = v.x;
    h[4 * q + 1] = v.y;
    h[4 * q + 2] = v.z;
    h[4 * q + 3] = v.w;
  }
}

template <typename TV>
struct KryArgs {
  int n, r, max_cluster, max_hnbr, reorth_passes;
  double Es, Ep, defl_tol;
  const int* c_off;
  const int* c_idx;
  const int* h_off;
  const int* h_idx;
  const TV* H;
  double* T;
  TV* Y;
  unsigned long long* colmask;
  TV* Vg;
  int* lcol;
  int* lblk;
  int* st;
};

__device__ __forceinline__ int find_slot(const int* cl, int nc, int b) {
  if (b == cl[0]) return 0;
  int lo = 1, hi = nc;
  while (lo < hi) {
    int mid = (lo + hi) >> 1;
    if (cl[mid] < b) lo = mid + 1; else hi = mid;
  }
  return (lo < nc && cl[lo] == b) ? lo : -1;
}

__host__ __device__ __forceinline__ size_t align16(size_t x) { return (x + 15) & ~size_t(15); }

template <typename TV>
__host__ __device__ inline size_t kry_smem_bytes(int r, int max_cluster, bool vsmem) {
  const size_t Dmax = 4 * (size_t)max_cluster;
  size_t b = 0;
  b += align16(sizeof(int) * max_cluster);            // cl
  b += align16(sizeof(int) * (max_cluster + 1));      // rowptr
  b += align16(sizeof(TV) * Dmax * 4);                // W
  if (vsmem) b += align16(sizeof(TV) * Dmax * 4 * r); // basis
  b += align16(sizeof(TV) * 16 * r);                  // projection coefficients
  b += align16(sizeof(TV) * 16 * 2);                  // A_k, B_{k-1}
  b += align16(sizeof(double) * 16);                  // B_k (FP64)
  b += align16(sizeof(TV) * 16 * KW);                 // reduction scratch
  b += align16(sizeof(int) * 16);                     // flags
  return b;
}

template <typename TV, bool VSMEM>
__global__ void __launch_bounds__(KT) krylov_kernel(const KryArgs<TV> a) {
  extern __shared__ __align__(16) unsigned char smem[];
  const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
  const int r = a.r, NT = 4 * r, Dmax = 4 * a.max_cluster;
  size_t off = 0;
  int* cl = reinterpret_cast<int*>(smem + off);      off += align16(sizeof(int) * a.max_cluster);
  int* rowptr = reinterpret_cast<int*>(smem + off);  off += align16(sizeof(int) * (a.max_cluster + 1));
  TV* W = reinterpret_cast<TV*>(smem + off);         off += align16(sizeof(TV) * Dmax * 4);
  TV* V;
  if (VSMEM) {
    V = reinterpret_cast<TV*>(smem + off);
    off += align16(sizeof(TV) * (size_t)Dmax * 4 * r);
  } else {
    V = a.Vg + (size_t)blockIdx.x * Dmax * 4 * r;
  }
  TV* Cc = reinterpret_cast<TV*>(smem + off);        off += align16(sizeof(TV) * 16 * r);
  TV* Ablk = reinterpret_cast<TV*>(smem + off);
  TV* Bp = Ablk + 16;                                off += align16(sizeof(TV) * 32);
  double* Bs = reinterpret_cast<double*>(smem + off); off += align16(sizeof(double) * 16);
  TV* red = reinterpret_cast<TV*>(smem + off);       off += align16(sizeof(TV) * 16 * KW);
  int* flags = reinterpret_cast<int*>(smem + off);
  int* lcol = a.lcol + (size_t)blockIdx.x * a.max_cluster * a.max_hnbr;
  int* lblk = a.lblk + (size_t)blockIdx.x * a.max_cluster * a.max_hnbr;
  const TV Es = (TV)a.Es, Ep = (TV)a.Ep;

  for (int i = blockIdx.x; i < a.n; i += gridDim.x) {
    const int c0 = a.c_off[i];
    const int nc = a.c_off[i + 1] - c0;
    double* Ti = a.T + (size_t)i * NT * NT;
    for (int q = tid; q < NT * NT; q += KT) Ti[q] = 0.0;
    const bool bad = (nc < 1 || nc > a.max_cluster || a.c_idx[c0] != i);
    if (bad) {
      if (tid == 0) {
        tbk::set_status(a.st, TB_ERR_INVALID_ARG, i);
        a.colmask[i] = 0ull;
      }
      __syncthreads();
      continue;
    }
    for (int s = tid; s < nc; s += KT) cl[s] = a.c_idx[c0 + s];
    const int deg = a.h_off[i + 1] - a.h_off[i];
    if (deg > a.max_hnbr) {            // lists longer than the capacity: refuse
      if (tid == 0) {
        tbk::set_status(a.st, TB_ERR_CAPACITY, deg);
        a.colmask[i] = 0ull;
      }
      __syncthreads();
      continue;
    }
    __syncthreads();
    // ---- local sparsity of H_c: counts, block-wide exclusive scan, fill
    for (int s = tid; s < nc; s += KT) {
      const int at = cl[s];
      int cnt = 0;
      const int pe = min(a.h_off[at + 1], a.h_off[at] + a.max_hnbr);
      for (int p = a.h_off[at]; p < pe; ++p)
        cnt += find_slot(cl, nc, a.h_idx[p]) >= 0;
      rowptr[s] = cnt;
    }
    __syncthreads();
    {
      int v[4], tot = 0;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = tid * 4 + q;
        v[q] = idx < nc ? rowptr[idx] : 0;
        tot += v[q];
      }
      int x = tot;
#pragma unroll
      for (int o = 1; o < 32; o <<= 1) {
        int y = __shfl_up_sync(0xffffffffu, x, o);
        if (lane >= o) x += y;
      }
      if (lane == 31) flags[warp] = x;
      __syncthreads();
      int wbase = 0;
      for (int w = 0; w < warp; ++w) wbase += flags[w];
      int run = wbase + x - tot;
#pragma unroll
      for (int q = 0; q < 4; ++q) {
        const int idx = tid * 4 + q;
        if (idx < nc) {
          rowptr[idx] = run;
          run += v[q];
          if (idx == nc - 1) rowptr[nc] = run;
        }
      }
      __syncthreads();
    }
    for (int s = tid; s < nc; s += KT) {
      const int at = cl[s];
      int e = rowptr[s];
      const int pe = min(a.h_off[at + 1], a.h_off[at] + a.max_hnbr);
      for (int p = a.h_off[at]; p < pe; ++p) {
        const int t = find_slot(cl, nc, a.h_idx[p]);
        if (t >= 0) {
          lcol[e] = t;
          lblk[e] = p;
          ++e;
        }
      }
    }
    // seed block V_1 = E_i
    const int D = 4 * nc;
    for (int q = tid; q < D * 4; q += KT) {
      const int row = q >> 2, c = q & 3;
      V[q] = (row == c) ? (TV)1 : (TV)0;
    }
    if (tid < 16) Bp[tid] = (TV)0;
    if (tid == 0) { flags[FL_MASK] = 0xF; flags[FL_MASK + 1] = 0; flags[FL_ACT] = 0xF; }
    __syncthreads();
    if (tid == 0 && rowptr[1] - rowptr[0] != deg) tbk::set_status(a.st, TB_ERR_INVALID_ARG, i);

    int nblocks = 1;
    for (int k = 0; k < r; ++k) {
      const TV* Vk = V + (size_t)k * Dmax * 4;
      const TV* Vp = V + (size_t)(k > 0 ? k - 1 : 0) * Dmax * 4;
      // ---- W = H_c V_k - V_{k-1} B_{k-1}^T
      for (int it = tid; it < 4 * nc; it += KT) {
        const int s = it >> 2, c = it & 3;
        TV x0 = Vk[(4 * s + 0) * 4 + c], x1 = Vk[(4 * s + 1) * 4 + c];
        TV x2 = Vk[(4 * s + 2) * 4 + c], x3 = Vk[(4 * s + 3) * 4 + c];
        TV a0 = Es * x0, a1 = Ep * x1, a2 = Ep * x2, a3 = Ep * x3;
        const int e1 = rowptr[s + 1];
        for (int e = rowptr[s]; e < e1; ++e) {
          const int t = lcol[e];
          TV h[16];
          load_h(a.H, lblk[e], h);
          const TV y0 = Vk[(4 * t + 0) * 4 + c], y1 = Vk[(4 * t + 1) * 4 + c];
          const TV y2 = Vk[(4 * t + 2) * 4 + c], y3 = Vk[(4 * t + 3) * 4 + c];
          a0 += h[0] * y0 + h[1] * y1 + h[2] * y2 + h[3] * y3;
          a1 += h[4] * y0 + h[5] * y1 + h[6] * y2 + h[7] * y3;
          a2 += h[8] * y0 + h[9] * y1 + h[10] * y2 + h[11] * y3;
          a3 += h[12] * y0 + h[13] * y1 + h[14] * y2 + h[15] * y3;
        }
        if (k > 0) {
          const TV b0 = Bp[c * 4 + 0], b1 = Bp[c * 4 + 1], b2 = Bp[c * 4 + 2], b3 = Bp[c * 4 + 3];
          const TV* pr = Vp + (4 * s) * 4;
          a0 -= pr[0] * b0 + pr[1] * b1 + pr[2] * b2 + pr[3] * b3;
          a1 -= pr[4] * b0 + pr[5] * b1 + pr[6] * b2 + pr[7] * b3;
          a2 -= pr[8] * b0 + pr[9] * b1 + pr[10] * b2 + pr[11] * b3;
          a3 -= pr[12] * b0 + pr[13] * b1 + pr[14] * b2 + pr[15] * b3;
        }
        W[(4 * s + 0) * 4 + c] = a0;
        W[(4 * s + 1) * 4 + c] = a1;
        W[(4 * s + 2) * 4 + c] = a2;
        W[(4 * s + 3) * 4 + c] = a3;
      }
      __syncthreads();
      // ---- A_k = V_k^T W
      {
        TV part[16];
#pragma unroll
        for (int q = 0; q < 16; ++q) part[q] = (TV)0;
        for (int row = tid; row < D; row += KT) {
          TV v[4], w[4];
#pragma unroll
          for (int q = 0; q < 4; ++q) { v[q] = Vk[row * 4 + q]; w[q] = W[row * 4 + q]; }
#pragma unroll
          for (int ii = 0; ii < 4; ++ii)
#pragma unroll
            for (int c = 0; c < 4; ++c) part[ii * 4 + c] += v[ii] * w[c];
        }
        tbk::block_sum<TV, 16>(part, red, Ablk);
      }
      if (tid < 16) {
        const int ii = tid >> 2, c = tid & 3;
        Ti[(4 * k + ii) * NT + 4 * k + c] = 0.5 * ((double)Ablk[ii * 4 + c] + (double)Ablk[c * 4 + ii]);
      }
      for (int row = tid; row < D; row += KT) {
        TV v[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) v[q] = Vk[row * 4 + q];
#pragma unroll
        for (int c = 0; c < 4; ++c)
          W[row * 4 + c] -= v[0] * Ablk[c] + v[1] * Ablk[4 + c] + v[2] * Ablk[8 + c] + v[3] * Ablk[12 + c];
      }
      __syncthreads();
      if (k == r - 1) break;
      // ---- full reorthogonalisation: classical Gram-Schmidt against V_1..V_k
      for (int pass = 0; pass < a.reorth_passes; ++pass) {
        for (int b = warp; b <= k; b += KW) {
          const TV* Vb = V + (size_t)b * Dmax * 4;
          TV part[16];
#pragma unroll
          for (int q = 0; q < 16; ++q) part[q] = (TV)0;
          for (int row = lane; row < D; row += 32) {
            TV v[4], w[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) { v[q] = Vb[row * 4 + q]; w[q] = W[row * 4 + q]; }
#pragma unroll
            for (int ii = 0; ii < 4; ++ii)
#pragma unroll
              for (int c = 0; c < 4; ++c) part[ii * 4 + c] += v[ii] * w[c];
          }
#pragma unroll
          for (int q = 0; q < 16; ++q) part[q] = tbk::warp_sum(part[q]);
          if (lane < 16) {
            TV val = part[0];
#pragma unroll
            for (int q = 1; q < 16; ++q) if (lane == q) val = part[q];
            Cc[b * 16 + lane] = val;
          }
        }
        __syncthreads();
        for (int row = tid; row < D; row += KT) {
          TV w[4];
#pragma unroll
          for (int c = 0; c < 4; ++c) w[c] = W[row * 4 + c];
          for (int b = 0; b <= k; ++b) {
            const TV* vb = V + (size_t)b * Dmax * 4 + row * 4;
            const TV v0 = vb[0], v1 = vb[1], v2 = vb[2], v3 = vb[3];
            const TV* cb = Cc + b * 16;
#pragma unroll
            for (int c = 0; c < 4; ++c)
              w[c] -= v0 * cb[c] + v1 * cb[4 + c] + v2 * cb[8 + c] + v3 * cb[12 + c];
          }
#pragma unroll
          for (int c = 0; c < 4; ++c) W[row * 4 + c] = w[c];
        }
        __syncthreads();
      }
      // ---- in-block QR with deflation (one warp): W = V_{k+1} B_k
      if (warp == 0) {
        TV* Vn = V + (size_t)(k + 1) * Dmax * 4;
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
              const TV w = W[row * 4 + c];
#pragma unroll
              for (int j = 0; j < 3; ++j) if (j < c) dd[j] += Vn[row * 4 + j] * w;
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) if (j < c) dd[j] = tbk::warp_sum(dd[j]);
            for (int row = lane; row < D; row += 32) {
              TV w = W[row * 4 + c];
#pragma unroll
              for (int j = 0; j < 3; ++j) if (j < c) w -= dd[j] * Vn[row * 4 + j];
              W[row * 4 + c] = w;
            }
#pragma unroll
            for (int j = 0; j < 3; ++j) if (j < c) R[j * 4 + c] += (double)dd[j];
          }
          TV nn = (TV)0;
          for (int row = lane; row < D; row += 32) {
            const TV w = W[row * 4 + c];
            nn += w * w;
          }
          nn = tbk::warp_sum(nn);
          const double nrm = sqrt((double)nn);
          if (!isfinite(nrm)) nonfinite = true;
          if (nrm > a.defl_tol) {
            const TV inv = (TV)(1.0 / nrm);
            for (int row = lane; row < D; row += 32) Vn[row * 4 + c] = W[row * 4 + c] * inv;
            R[c * 4 + c] = nrm;
            act |= 1 << c;
          } else {
            for (int row = lane; row < D; row += 32) Vn[row * 4 + c] = (TV)0;
          }
        }
        if (lane == 0) {
#pragma unroll
          for (int q = 0; q < 16; ++q) Bs[q] = R[q];
#pragma unroll
          for (int j = 0; j < 4; ++j)
#pragma unroll
            for (int c = 0; c < 4; ++c) {
              Ti[(4 * (k + 1) + j) * NT + 4 * k + c] = R[j * 4 + c];
              Ti[(4 * k + c) * NT + 4 * (k + 1) + j] = R[j * 4 + c];
            }
          flags[FL_ACT] = act;
          // active-column mask of the basis, 64 bits kept as two ints
          unsigned long long mask = ((unsigned long long)(unsigned)flags[FL_MASK + 1] << 32) |
                                    (unsigned)flags[FL_MASK];
          mask |= (unsigned long long)act << (4 * (k + 1));
          flags[FL_MASK] = (int)(mask & 0xffffffffull);
          flags[FL_MASK + 1] = (int)(mask >> 32);
          if (nonfinite) tbk::set_status(a.st, TB_ERR_NONFINITE, i);
        }
      }
      __syncthreads();
      if (tid < 16) Bp[tid] = (TV)Bs[tid];
      const int act_now = flags[FL_ACT];
      __syncthreads();
      if (act_now == 0) break;
      nblocks = k + 2;
    }
    // ---- outputs: column mask, rows of V for the target and its H neighbours
    if (tid == 0)
      a.colmask[i] = ((unsigned long long)(unsigned)flags[FL_MASK + 1] << 32) | (unsigned)flags[FL_MASK];
    {
      const size_t ybase = (size_t)(i + a.h_off[i]) * 4;
      const int nrows = (deg + 1) * 4;
      for (int q = tid; q < nrows * NT; q += KT) {
        const int rr = q / NT, col = q - rr * NT;
        const int qq = rr >> 2, beta = rr & 3;
        const int slot = qq == 0 ? 0 : lcol[rowptr[0] + qq - 1];
        const int b = col >> 2, c = col & 3;
        TV val = (TV)0;
        if (b < nblocks) val = V[(size_t)b * Dmax * 4 + (4 * slot + beta) * 4 + c];
        a.Y[(ybase + rr) * NT + col] = val;
      }
    }
    __syncthreads();
  }
}

template <typename TV, bool VSMEM>
tb_status launch_t(tb_ctx* c, int n, const int* c_off, const int* c_idx, const int* h_off,
                   const int* h_idx, const TV* H, cudaStream_t s) {
  const tb_params& p = c->p;
  KryArgs<TV> a;
  a.n = n; a.r = p.r; a.max_cluster = p.max_cluster; a.max_hnbr = p.max_hnbr;
  a.reorth_passes = p.reorth_passes;
  a.Es = p.Es; a.Ep = p.Ep; a.defl_tol = p.defl_tol;
  a.c_off = c_off; a.c_idx = c_idx; a.h_off = h_off; a.h_idx = h_idx; a.H = H;
  a.T = c->T; a.Y = reinterpret_cast<TV*>(c->Y); a.colmask = c->colmask;
  a.Vg = reinterpret_cast<TV*>(c->Vg); a.lcol = c->lcol; a.lblk = c->lblk; a.st = c->d_status;
  const int grid = n < c->kry_grid ? n : c->kry_grid;
  if (grid <= 0) return TB_OK;
  krylov_kernel<TV, VSMEM><<<grid, KT, c->kry_smem, s>>>(a);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}

template <typename TV, bool VSMEM>
tb_status configure_t(tb_ctx* c, int max_smem) {
  const size_t bytes = kry_smem_bytes<TV>(c->p.r, c->p.max_cluster, VSMEM);
  if ((int)bytes > max_smem) return TB_ERR_CAPACITY;
  TB_CUDA_TRY(cudaFuncSetAttribute(krylov_kernel<TV, VSMEM>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bytes));
  int occ = 0;
  TB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, krylov_kernel<TV, VSMEM>,
                                                            KT, bytes));
  if (occ < 1) return TB_ERR_CAPACITY;
  c->kry_smem = bytes;
  c->kry_vsmem = VSMEM;
  c->kry_grid = c->num_sms * occ;
  return TB_OK;
}

}  // namespace

size_t krylov_basis_bytes_global(const tb_ctx* c) {
  if (c->kry_vsmem) return 0;
  const size_t tv = c->p.prec == TB_PREC_FP64 ? sizeof(double) : sizeof(float);
  return (size_t)c->kry_grid * 4 * c->p.max_cluster * 4 * c->p.r * tv;
}

tb_status krylov_configure(tb_ctx* c) {
  int dev = 0, max_smem = 0;
  TB_CUDA_TRY(cudaGetDevice(&dev));
  TB_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const bool force_global = getenv("TB_KRYLOV_BASIS_GLOBAL") != nullptr;
  if (c->p.prec == TB_PREC_FP64) {
    if (!force_global && configure_t<double, true>(c, max_smem) == TB_OK) return TB_OK;
    return configure_t<double, false>(c, max_smem);
  }
  if (!force_global && configure_t<float, true>(c, max_smem) == TB_OK) return TB_OK;
  return configure_t<float, false>(c, max_smem);
}

tb_status launch_krylov(tb_ctx* c, int n, const int* c_off, const int* c_idx,
                        const int* h_off, const int* h_idx, const double* Hblk,
                        const float* Hmir, cudaStream_t s) {
  if (c->p.prec == TB_PREC_FP64) {
    if (c->kry_vsmem) return launch_t<double, true>(c, n, c_off, c_idx, h_off, h_idx, Hblk, s);
    return launch_t<double, false>(c, n, c_off, c_idx, h_off, h_idx, Hblk, s);
  }
  if (!Hmir) return TB_ERR_INVALID_ARG;
  if (c->kry_vsmem) return launch_t<float, true>(c, n, c_off, c_idx, h_off, h_idx, Hmir, s);
  return launch_t<float, false>(c, n, c_off, c_idx, h_off, h_idx, Hmir, s);
}
