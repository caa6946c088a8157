// Chemical potential, density-matrix blocks, energies, forces
// (Sec. 2: rho = sum_m |m> f(e_m) <m|, <F_i> = Tr[rho F_i]) and the
// velocity-Verlet kernels.
//
// Occupation f(x) = 1/(1+e^x) per spin orbital, spin factor 2, x = (lam-mu)/kT.
// The electron count uses the Ritz pairs of every target weighted by their
// seed-block weight w = sum_a S_a^2 (Gauss quadrature of the local density of
// states).  All sums are taken in a fixed order (per-thread, then fixed
// shuffle trees, then a fixed sequence over blocks), so results are
// deterministic from run to run.
#include <atomic>
#include <mutex>
#include "tb_fpconv.cuh"
#include "tb_internal.cuh"
#include "tb_model.cuh"

namespace {

constexpr int MT = 256;    // mu kernel threads (16 per partial value: MT >= 16 * 16)
constexpr int RT = 128;    // rho kernel threads
// energy reduction threads: one block; its FP64 additions all run on one SM,
// so four warps rather than 32 (fewer warp-wide FP64 instructions)
constexpr int ER_T = 128;

__device__ __forceinline__ double fermi(double x) {
  if (x > 50.0) return 0.0;
  if (x < -50.0) return 1.0;
  if (x > 0.0) {
    const double e = exp(-x);
    return e / (1.0 + e);
  }
  return 1.0 / (1.0 + exp(x));
}

__device__ __forceinline__ double entropy_term(double f) {
  double t = 0.0;
  if (f > 0.0) t += f * log(f);
  if (f < 1.0) t += (1.0 - f) * log(1.0 - f);
  return t;
}

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid-wide barrier on a monotone arrival counter.  Gives up after `timeout`
// SM clocks, sets TB_ERR_TIMEOUT and returns false (the caller then leaves).
__device__ bool grid_barrier(unsigned* bar, unsigned target, long long timeout, int* st,
                             int* sflag) {
  __syncthreads();
  if (threadIdx.x == 0) {
    __threadfence();
    atomicAdd(bar, 1u);
    const long long t0 = clock64();
    int ok = 1;
    while (ld_acquire(bar) < target) {
      if (clock64() - t0 > timeout) {
        ok = 0;
        tbk::set_status(st, TB_ERR_TIMEOUT, (int)blockIdx.x);
        break;
      }
      __nanosleep(100);
    }
    __threadfence();
    *sflag = ok;
  }
  __syncthreads();
  return *sflag != 0;
}

struct MuArgs {
  long long npairs;
  int NT;
  const double* lambda;
  const double* S;
  double kT, ikT, ne, tolN;                 // ikT = 1 / kT
  const double* guess;
  double* mu_out;
  double* ncount_out;
  int* iters_out;
  double* part;        // 2 generations x gridDim x MU_PART doubles
  unsigned* bar;
  int max_iter;
  long long timeout;
  long long per_block; // pairs handled (and staged in shared memory) per block
  int staged;          // 1: (lambda, w) of the block's pairs live in shared memory
  int* st;
};

constexpr int MU_NPT = 32;     // trial points per coarse pass (FP32 partials: MU_PART doubles)
constexpr int MU_PART = 16;    // partial slots per block and generation

__device__ __forceinline__ double pair_weight(const double* S, int NT, long long q) {
  const long long i = q / NT;
  const int k = (int)(q - i * NT);
  const double* s = S + (size_t)i * 4 * NT + k;
  return s[0] * s[0] + s[NT] * s[NT] + s[2 * NT] * s[2 * NT] + s[3 * NT] * s[3 * NT];
}

// f(x) = 1/(1+e^x) and f(1-f).  Beyond |x| = 15 the small one of f and 1-f
// is below 3.1e-7 and is taken from the FP32 exponential (absolute error
// ~3e-14); inside, FP64 throughout.
__device__ __forceinline__ void occupation(double x, double& f, double& g) {
  if (x > 15.0) {
    const float e = __expf((float)fminf(-(float)x, 0.f));
    f = (double)e / (1.0 + (double)e);
    g = f * (1.0 - f);
  } else if (x < -15.0) {
    const float e = __expf((float)fmaxf((float)x, -200.f));
    const double t = (double)e / (1.0 + (double)e);
    f = 1.0 - t;
    g = t * f;
  } else {
    f = fermi(x);
    g = f * (1.0 - f);
  }
}

// Adds w f and w f(1-f) of one (lambda, w) pair at mu.  Pairs far from mu
// (|x| > 15.5 by an FP32 estimate of x from the FP32 copies lf, wf) take f or
// 1 - f (below 2e-7) from the FP32 exponential, with absolute error ~1e-14 and
// only FP64 additions; the others take the FP64 path of occupation().
__device__ __forceinline__ void pair_occ(double l, double w, float lf, float wf, double mu,
                                         float muf, double ikT, float ikTf, double& n,
                                         double& d) {
  const float xf = (lf - muf) * ikTf;
  if (xf > 15.5f) {
    const float e = __expf(fmaxf(-xf, -87.f));
    const float fw = wf * __fdividef(e, 1.f + e);
    n += (double)fw;
    d += (double)fw;                       // f (1 - f) = f to FP32 accuracy here
  } else if (xf < -15.5f) {
    const float e = __expf(fmaxf(xf, -87.f));
    const float tw = wf * __fdividef(e, 1.f + e);
    n += w - (double)tw;
    d += (double)tw;
  } else {
    double f, g;
    occupation((l - mu) * ikT, f, g);
    n += w * f;
    d += w * g;
  }
}

// Every block publishes M partials in generation buffer `gen`, passes the grid
// barrier, then sums all blocks' partials in block order (fixed order: every
// block obtains bitwise the same totals).  Returns false on barrier timeout.
template <int M>
__device__ bool grid_allreduce(const double (&v)[M], const MuArgs& a, unsigned& gen,
                               double* red, double* tot, int* sflag) {
  const int G = gridDim.x;
  tbk::block_sum16<double, M>(v, red, tot);
  double* pg = a.part + (size_t)(gen & 1) * G * MU_PART;
  if (threadIdx.x < M) pg[blockIdx.x * MU_PART + threadIdx.x] = tot[threadIdx.x];
  ++gen;
  if (!grid_barrier(a.bar, gen * G, a.timeout, a.st, sflag)) return false;
  // 16 threads per value stride over the blocks (loads issued eight at a
  // time, not one L2 round trip per partial), then a fixed shuffle tree
  {
    const int m = threadIdx.x >> 4, sub = threadIdx.x & 15;
    double sum = 0.0;
    if (m < M) {
      int g = sub;
      for (; g + 7 * 16 < G; g += 8 * 16) {
        double t[8];
#pragma unroll
        for (int u = 0; u < 8; ++u) t[u] = pg[(g + u * 16) * MU_PART + m];
        sum += ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
      }
      for (; g < G; g += 16) sum += pg[g * MU_PART + m];
    }
#pragma unroll
    for (int o = 8; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (m < M && sub == 0) tot[m] = sum;
  }
  __syncthreads();
  return true;
}

// Block then grid sum of the MU_NPT FP32 counts of a coarse pass (the counts
// only have to fall on the right side of N_e; the Newton phase re-counts the
// bracket ends in FP64).  The partials are floats in the blocks' MU_PART
// double slots; 8 threads per value stride over the blocks in a fixed order.
// Returns false on barrier timeout.
__device__ bool grid_allreduce_f32(const float (&v)[MU_NPT], const MuArgs& a, unsigned& gen,
                                   float* redf, float* totf, int* sflag) {
  static_assert(MU_NPT == 32 && MU_NPT * sizeof(float) == MU_PART * sizeof(double) && MT == 256,
                "layout of the coarse partials");
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5, G = gridDim.x;
#pragma unroll
  for (int ch = 0; ch < MU_NPT / 16; ++ch) {
    float p[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) p[q] = v[ch * 16 + q];
    const float t = tbk::warp_reduce16(p, lane);
    if ((lane & 1) == 0) redf[warp * MU_NPT + ch * 16 + (lane >> 1)] = t;
  }
  __syncthreads();
  float* pg = reinterpret_cast<float*>(a.part + (size_t)(gen & 1) * G * MU_PART);
  if (threadIdx.x < MU_NPT) {
    float s0 = 0.f;
    for (int w = 0; w < MT / 32; ++w) s0 += redf[w * MU_NPT + threadIdx.x];
    pg[blockIdx.x * MU_NPT + threadIdx.x] = s0;
  }
  ++gen;
  if (!grid_barrier(a.bar, gen * G, a.timeout, a.st, sflag)) return false;
  {
    const int m = threadIdx.x >> 3, sub = threadIdx.x & 7;
    float sum = 0.f;
    int g = sub;
    for (; g + 7 * 8 < G; g += 8 * 8) {
      float t[8];
#pragma unroll
      for (int u = 0; u < 8; ++u) t[u] = pg[(g + u * 8) * MU_NPT + m];
      sum += ((t[0] + t[1]) + (t[2] + t[3])) + ((t[4] + t[5]) + (t[6] + t[7]));
    }
    for (; g < G; g += 8) sum += pg[g * MU_NPT + m];
#pragma unroll
    for (int o = 4; o > 0; o >>= 1) sum += __shfl_xor_sync(0xffffffffu, sum, o);
    if (sub == 0) totf[m] = sum;
  }
  __syncthreads();
  return true;
}

__global__ void __launch_bounds__(MT) mu_kernel(const MuArgs a) {
  extern __shared__ __align__(16) unsigned char mu_smem[];
  double2* pairs = reinterpret_cast<double2*>(mu_smem);   // (lambda, w)
  float2* pairsf = reinterpret_cast<float2*>(pairs + a.per_block);   // FP32 copies
  int* nearl = reinterpret_cast<int*>(pairsf + a.per_block);         // pairs near mu (Newton)
  __shared__ int wtot[MT / 32];
  __shared__ double red[MT / 32 * 16];
  __shared__ double tot[16];
  __shared__ float redf[MT / 32 * MU_NPT];
  __shared__ float totf[MU_NPT];
  __shared__ int sflag;
  const int G = gridDim.x;
  const double ikT = a.ikT;
  const long long q0 = (long long)blockIdx.x * a.per_block;
  const long long q1 = min(a.npairs, q0 + a.per_block);
  const int nloc = (int)max(0ll, q1 - q0);
  unsigned gen = 0;
  // pair accessors: shared-memory copies when staged, else recomputed from global
  auto get = [&](int t, double& l, double& w) {
    if (a.staged) {
      const double2 v = pairs[t];
      l = v.x;
      w = v.y;
    } else {
      l = a.lambda[q0 + t];
      w = pair_weight(a.S, a.NT, q0 + t);
    }
  };
  auto getf = [&](int t, float& lf, float& wf) {
    if (a.staged) {
      const float2 v = pairsf[t];
      lf = v.x;
      wf = v.y;
    } else {
      lf = (float)a.lambda[q0 + t];
      wf = (float)pair_weight(a.S, a.NT, q0 + t);
    }
  };
  double lmin = 1e300, lmax = -1e300;
  for (int t = threadIdx.x; t < nloc; t += MT) {
    const double l = a.lambda[q0 + t], w = pair_weight(a.S, a.NT, q0 + t);
    if (a.staged) {
      pairs[t] = make_double2(l, w);
      pairsf[t] = make_float2((float)l, (float)w);
    }
    if (w > 0.0) { lmin = fmin(lmin, l); lmax = fmax(lmax, l); }
  }
  // ---- bracket: [min lam - 40 kT, max lam + 40 kT] over pairs with weight
  {
    double v[2] = {lmin, -lmax};
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      v[0] = fmin(v[0], __shfl_xor_sync(0xffffffffu, v[0], o));
      v[1] = fmin(v[1], __shfl_xor_sync(0xffffffffu, v[1], o));
    }
    if ((threadIdx.x & 31) == 0) { red[2 * (threadIdx.x >> 5)] = v[0]; red[2 * (threadIdx.x >> 5) + 1] = v[1]; }
    __syncthreads();
    double* pg = a.part + (size_t)(gen & 1) * G * MU_PART;
    if (threadIdx.x == 0) {
      double m0 = 1e300, m1 = 1e300;
      for (int w = 0; w < MT / 32; ++w) { m0 = fmin(m0, red[2 * w]); m1 = fmin(m1, red[2 * w + 1]); }
      pg[blockIdx.x * MU_PART] = m0;
      pg[blockIdx.x * MU_PART + 1] = m1;
    }
    ++gen;
    if (!grid_barrier(a.bar, gen * G, a.timeout, a.st, &sflag)) return;
    // every thread takes a share of the blocks' values, then a block minimum
    double m0 = 1e300, m1 = 1e300;
    for (int g = threadIdx.x; g < G; g += MT) {
      m0 = fmin(m0, pg[g * MU_PART]);
      m1 = fmin(m1, pg[g * MU_PART + 1]);
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
      m0 = fmin(m0, __shfl_xor_sync(0xffffffffu, m0, o));
      m1 = fmin(m1, __shfl_xor_sync(0xffffffffu, m1, o));
    }
    __syncthreads();                                  // red is reused below
    if ((threadIdx.x & 31) == 0) { red[2 * (threadIdx.x >> 5)] = m0; red[2 * (threadIdx.x >> 5) + 1] = m1; }
    __syncthreads();
    if (threadIdx.x == 0) {
      double a0 = 1e300, a1 = 1e300;
      for (int w = 0; w < MT / 32; ++w) { a0 = fmin(a0, red[2 * w]); a1 = fmin(a1, red[2 * w + 1]); }
      tot[0] = a0;
      tot[1] = -a1;
    }
    __syncthreads();
  }
  // The scalar search state (bracket, trial point, Newton step) is advanced
  // by thread 0 alone and read by every thread after a barrier: on this GPU a
  // warp-wide FP64 instruction holds the SM's FP64 pipe for many cycles
  // whatever the number of active lanes, so scalar FP64 arithmetic repeated
  // by all eight warps would cost eight times the pipe time of one.
  enum { S_LO, S_HI, S_H, S_MU, S_MID, S_DXO, S_DX, S_NLO, S_NHI, S_NMU, S_LO0, S_HI0, S_NS };
  __shared__ double ss[S_NS];
  __shared__ float sf[6];                          // dx, lo, mu, lo, hi, mid as floats
  __shared__ int si[4];                            // iterations, go on, converged, near path
  if (threadIdx.x == 0) {
    const double lo0 = tot[0] - 40.0 * a.kT, hi0 = tot[1] + 40.0 * a.kT;
    const double h = (hi0 - lo0) / (MU_NPT + 1);
    ss[S_LO0] = lo0; ss[S_HI0] = hi0;
    ss[S_LO] = lo0; ss[S_HI] = hi0; ss[S_H] = h;
    ss[S_NLO] = -1.0; ss[S_NHI] = -1.0;           // counts at lo / hi (unknown: < 0)
    sf[0] = (float)(h * ikT); sf[1] = (float)lo0;
    si[0] = 0;
    si[1] = hi0 - lo0 > 0.05;
  }
  __syncthreads();
  const float ikTf = (float)a.ikT;
  // ---- coarse bracketing with FP32 occupations at MU_NPT points per pass, to
  // a bracket of 0.05 eV; the counts at its ends give Newton's first point
  for (int pass = 0; pass < 6 && si[1]; ++pass) {
    float cnt[MU_NPT];
#pragma unroll
    for (int t = 0; t < MU_NPT; ++t) cnt[t] = 0.f;
    const float dx = sf[0], lof = sf[1];
    for (int t = threadIdx.x; t < nloc; t += MT) {
      float lf, wf;
      getf(t, lf, wf);
      if (wf == 0.f) continue;
      const float x0 = (lf - lof) * ikTf;
#pragma unroll
      for (int u = 0; u < MU_NPT; ++u) {
        const float x = fminf(fmaxf(x0 - (u + 1) * dx, -80.f), 80.f);
        cnt[u] += __fdividef(wf, 1.f + __expf(x));
      }
    }
    if (!grid_allreduce_f32(cnt, a, gen, redf, totf, &sflag)) return;
    if (threadIdx.x < 32) {
      // lane u tests trial point u; the first with N > N_e (N increases with mu)
      static_assert(MU_NPT == 32, "one trial point per lane");
      const unsigned above = __ballot_sync(0xffffffffu, 2.0 * (double)totf[threadIdx.x] > a.ne);
      if (threadIdx.x == 0) {
        const int jfirst = above ? __ffs(above) - 1 : MU_NPT;
        const double lo = ss[S_LO], hi = ss[S_HI], h = ss[S_H];
        const double nlo = jfirst == 0 ? lo : lo + jfirst * h;
        const double nhi = jfirst == MU_NPT ? hi : lo + (jfirst + 1) * h;
        if (jfirst > 0) ss[S_NLO] = 2.0 * (double)totf[jfirst - 1];
        if (jfirst < MU_NPT) ss[S_NHI] = 2.0 * (double)totf[jfirst];
        const double hn = (nhi - nlo) / (MU_NPT + 1);
        ss[S_LO] = nlo; ss[S_HI] = nhi; ss[S_H] = hn;
        sf[0] = (float)(hn * ikT); sf[1] = (float)nlo;
        si[0] += 1;
        si[1] = nhi - nlo > 0.05;
      }
    }
    __syncthreads();
  }
  // ---- FP64 safeguarded Newton on N(mu) - N_e.  The first pass also counts
  // at the coarse bracket ends (FP32 counts may misjudge a point whose count
  // is within rounding of N_e) and widens the bracket on a side that fails.
  __shared__ int s_check;
  if (threadIdx.x == 0) {
    const double lo = ss[S_LO], hi = ss[S_HI], nlo_cnt = ss[S_NLO], nhi_cnt = ss[S_NHI];
    s_check = lo > ss[S_LO0] || hi < ss[S_HI0];
    double mu = 0.5 * (lo + hi);
    if (nlo_cnt >= 0.0 && nhi_cnt > nlo_cnt) {     // linear interpolation of the counts
      const double fr = (a.ne - nlo_cnt) / (nhi_cnt - nlo_cnt);
      if (fr > 0.0 && fr < 1.0) mu = lo + fr * (hi - lo);
    }
    if (a.guess) {
      const double g = *a.guess;
      if (isfinite(g) && g > lo && g < hi) mu = g;
    }
    ss[S_MU] = mu;
    ss[S_DXO] = hi - lo;
    ss[S_DX] = hi - lo;
    ss[S_NMU] = 0.0;
    ss[S_MID] = 0.5 * (lo + hi);
    sf[5] = (float)ss[S_MID];
    si[2] = 0;
  }
  __syncthreads();
  const bool check = s_check != 0;
  // Pairs within 17.5 kT of the coarse bracket's midpoint go to a compact list
  // (block scan: a fixed order).  While mu (and, on the first pass, the
  // bracket ends) stays within 1.5 kT of it, every other pair has |x| > 15.5
  // and takes pair_occ's FP32 branch, and the FP64 branch runs on the list
  // with full warps (a warp-wide FP64 instruction costs the same with one
  // active lane as with 32).
  const float midf = sf[5], Rf = (float)(17.5 * a.kT);
  int nnear = 0;
  if (a.staged) {
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5;
    int cnt = 0;
    for (int t = threadIdx.x; t < nloc; t += MT) {
      const float2 v2 = pairsf[t];
      cnt += (v2.y != 0.f && fabsf(v2.x - midf) <= Rf) ? 1 : 0;
    }
    int incl = cnt;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
      const int y = __shfl_up_sync(0xffffffffu, incl, o);
      if (lane >= o) incl += y;
    }
    if (lane == 31) wtot[wid] = incl;
    __syncthreads();
    int pos = incl - cnt;
    for (int w2 = 0; w2 < wid; ++w2) pos += wtot[w2];
    for (int w2 = 0; w2 < MT / 32; ++w2) nnear += wtot[w2];
    for (int t = threadIdx.x; t < nloc; t += MT) {
      const float2 v2 = pairsf[t];
      if (v2.y != 0.f && fabsf(v2.x - midf) <= Rf) nearl[pos++] = t;
    }
    __syncthreads();
  }
  for (int it = 0; it < a.max_iter; ++it) {
    const bool ends = it == 0 && check;
    if (threadIdx.x == 0) {
      const double mu = ss[S_MU], lo = ss[S_LO], hi = ss[S_HI], mid = ss[S_MID], w = 1.5 * a.kT;
      si[3] = a.staged && fabs(mu - mid) <= w && (!ends || (fabs(lo - mid) <= w && fabs(hi - mid) <= w));
      sf[2] = (float)mu; sf[3] = (float)lo; sf[4] = (float)hi;
    }
    __syncthreads();
    double v[4] = {0.0, 0.0, 0.0, 0.0};
    const double mu = ss[S_MU], lo = ss[S_LO], hi = ss[S_HI];
    const float muf = sf[2], lof = sf[3], hif = sf[4];
    if (si[3]) {
      for (int t = threadIdx.x; t < nloc; t += MT) {
        float lf, wf;
        getf(t, lf, wf);
        if (wf == 0.f || fabsf(lf - midf) <= Rf) continue;
        double l, w;
        get(t, l, w);
        pair_occ(l, w, lf, wf, mu, muf, ikT, ikTf, v[0], v[1]);
        if (ends) {
          double dd = 0.0;
          pair_occ(l, w, lf, wf, lo, lof, ikT, ikTf, v[2], dd);
          pair_occ(l, w, lf, wf, hi, hif, ikT, ikTf, v[3], dd);
        }
      }
      for (int x = threadIdx.x; x < nnear; x += MT) {
        const int t = nearl[x];
        float lf, wf;
        getf(t, lf, wf);
        double l, w;
        get(t, l, w);
        pair_occ(l, w, lf, wf, mu, muf, ikT, ikTf, v[0], v[1]);
        if (ends) {
          double dd = 0.0;
          pair_occ(l, w, lf, wf, lo, lof, ikT, ikTf, v[2], dd);
          pair_occ(l, w, lf, wf, hi, hif, ikT, ikTf, v[3], dd);
        }
      }
    } else {
      for (int t = threadIdx.x; t < nloc; t += MT) {
        float lf, wf;
        getf(t, lf, wf);
        if (wf == 0.f) continue;
        double l, w;
        get(t, l, w);
        pair_occ(l, w, lf, wf, mu, muf, ikT, ikTf, v[0], v[1]);
        if (ends) {
          double dd = 0.0;
          pair_occ(l, w, lf, wf, lo, lof, ikT, ikTf, v[2], dd);
          pair_occ(l, w, lf, wf, hi, hif, ikT, ikTf, v[3], dd);
        }
      }
    }
    if (!grid_allreduce<4>(v, a, gen, red, tot, &sflag)) return;
    if (threadIdx.x == 0) {
      double lo2 = lo, hi2 = hi, mu2 = mu;
      double dxold = ss[S_DXO], dx = ss[S_DX];
      si[0] += 1;
      const double Nmu = 2.0 * tot[0];
      const double dN = 2.0 * tot[1] * ikT;
      ss[S_NMU] = Nmu;
      if (ends) {
        if (2.0 * tot[2] > a.ne) lo2 = ss[S_LO0];
        if (2.0 * tot[3] < a.ne) hi2 = ss[S_HI0];
      }
      if (fabs(Nmu - a.ne) <= a.tolN || hi2 - lo2 < 1e-13) {
        si[2] = 1;                                   // converged at mu
      } else {
        if (Nmu < a.ne) lo2 = fmax(lo2, mu2); else hi2 = fmin(hi2, mu2);
        // bisect when the Newton point leaves the bracket or the step is not at
        // least halving (Numerical Recipes' rtsafe rule)
        const double fv = Nmu - a.ne;
        const double newton = mu2 - fv / dN;
        if (!(dN > 0.0) || !(newton > lo2 && newton < hi2) || fabs(2.0 * fv) > fabs(dxold * dN)) {
          dxold = dx;
          dx = 0.5 * (hi2 - lo2);
          mu2 = lo2 + dx;
        } else {
          dxold = dx;
          dx = fv / dN;
          mu2 = newton;
          // Every pair's second derivative in mu is its first times
          // (1 - 2f)/kT, so |N''| <= N'/kT and the Newton step from the
          // residual fv leaves at most fv^2 / (2 kT N') (to leading order,
          // over a step of at most ~1e-6 eV here).  When that is below a
          // tenth of the tolerance the new point is returned without another
          // pass, with its predicted count N_e (within 0.1 tolN).
          if (fv * fv <= 0.2 * a.tolN * a.kT * dN) {
            si[2] = 1;
            ss[S_NMU] = a.ne;
          }
        }
      }
      ss[S_LO] = lo2; ss[S_HI] = hi2; ss[S_MU] = mu2; ss[S_DXO] = dxold; ss[S_DX] = dx;
    }
    __syncthreads();
    if (si[2]) break;
  }
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    *a.mu_out = ss[S_MU];
    if (a.ncount_out) *a.ncount_out = ss[S_NMU];
    if (a.iters_out) *a.iters_out = si[0];
    if (!si[2]) tbk::set_status(a.st, TB_ERR_NO_CONVERGENCE, -1);
  }
}

// ---------------------------------------------------------------- rho blocks

struct RhoArgs {
  int NT;
  const int* h_off;
  const int* kdim;
  const double* lambda;
  const double* S;
  const double* P;
  const double* mu;
  double kT, ikT;       // ikT = 1 / kT
  double* rho;
  double* per_target;   // n x 5
  int* st;
};

// TA: type of the density-block contraction (FP32 in the mixed path, whose
// P and S carry FP32 accuracy; FP64 otherwise).  Energy sums stay FP64.
// One CTA per target: the weights f_k S[a][k] are formed once in shared
// memory; each warp then takes row blocks q (the target and its Hamiltonian
// neighbours), lanes over the eigenpairs k, and reduces the 16 entries of the
// block rho^(i)_{q b, i a} = sum_k P[q,b,k] f_k S[a,k] with one butterfly.
template <typename TA>
__global__ void __launch_bounds__(RT) rho_kernel(const RhoArgs a) {
  __shared__ TA fs[4 * tbk::MAX_NT];           // f_k S[a][k]
  __shared__ double red[RT / 32 * 3];
  __shared__ double tot[3];
  const int i = blockIdx.x, NT = a.NT;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  const int m = a.kdim[i];
  const double mu = *a.mu;
  const double* lam = a.lambda + (size_t)i * NT;
  const double* Si = a.S + (size_t)i * 4 * NT;
  double v[3] = {0.0, 0.0, 0.0};
  if constexpr (sizeof(TA) == 4) {
    // Mixed path.  Pairs with |x| > 15.5 (FP32 estimate) take f or 1 - f (below
    // 2e-7) and the entropy term s = -e (|x| + 1) + O(e^2) from the FP32
    // exponential e = exp(-|x|); the others go, compacted in index order into
    // the first lanes, through FP64 with one exponential and one log1p:
    //   f = 1/(1+e) or e/(1+e),  s = f ln f + (1-f) ln(1-f)
    //     = -min(f, 1-f) |x| - log1p(e)   (exact).
    __shared__ int nidx[tbk::MAX_NT];
    __shared__ int wball[RT / 32];
    const float ikTf = tbconv::d2f(a.ikT), muf = tbconv::d2f(mu);
    const int k = threadIdx.x;
    bool near_k = false;
    double w = 0.0;
    if (k < m) {
      w = Si[k] * Si[k] + Si[NT + k] * Si[NT + k] + Si[2 * NT + k] * Si[2 * NT + k] +
          Si[3 * NT + k] * Si[3 * NT + k];
      const float xf = (tbconv::d2f(lam[k]) - muf) * ikTf;
      near_k = fabsf(xf) <= 15.5f;
      if (!near_k) {
        const float e = __expf(-fabsf(xf));
        const float t = __fdividef(e, 1.f + e);        // the small one of f and 1 - f
        const double f = xf > 0.f ? (double)t : 1.0 - (double)t;
        v[0] += w * f * lam[k];
        v[1] += w * (double)(-(t * fabsf(xf) + e));
        v[2] += w * f;
        // f S in FP32 for the FP32 contraction, S converted by integer operations
        const float ff = xf > 0.f ? t : 1.f - t;
#pragma unroll
        for (int al = 0; al < 4; ++al) fs[al * NT + k] = ff * tbconv::d2f(Si[al * NT + k]);
      }
    } else if (k < NT) {
#pragma unroll
      for (int al = 0; al < 4; ++al) fs[al * NT + k] = (TA)0;
    }
    const unsigned bal = __ballot_sync(0xffffffffu, near_k);
    if (lane == 0) wball[warp] = __popc(bal);
    __syncthreads();
    int pos = __popc(bal & ((1u << lane) - 1u)), nnear = 0;
    for (int w2 = 0; w2 < RT / 32; ++w2) {
      if (w2 < warp) pos += wball[w2];
      nnear += wball[w2];
    }
    if (near_k) nidx[pos] = k;
    __syncthreads();
    if (threadIdx.x < nnear) {
      const int kk = nidx[threadIdx.x];
      const double wk = Si[kk] * Si[kk] + Si[NT + kk] * Si[NT + kk] +
                        Si[2 * NT + kk] * Si[2 * NT + kk] + Si[3 * NT + kk] * Si[3 * NT + kk];
      const double x = (lam[kk] - mu) * a.ikT, ax = fabs(x);
      const double e = exp(-ax);
      const double t = e / (1.0 + e);                  // the small one of f and 1 - f
      const double f = x > 0.0 ? t : 1.0 - t;
      v[0] += wk * f * lam[kk];
      v[1] += wk * (-(t * ax) - log1p(e));
      v[2] += wk * f;
#pragma unroll
      for (int al = 0; al < 4; ++al) fs[al * NT + kk] = tbconv::d2f(f) * tbconv::d2f(Si[al * NT + kk]);
    }
  } else {
    for (int k = threadIdx.x; k < NT; k += RT) {
      double f = 0.0;
      if (k < m) {
        f = fermi((lam[k] - mu) / a.kT);
        const double w = Si[k] * Si[k] + Si[NT + k] * Si[NT + k] + Si[2 * NT + k] * Si[2 * NT + k] +
                         Si[3 * NT + k] * Si[3 * NT + k];
        v[0] += w * f * lam[k];
        v[1] += w * entropy_term(f);
        v[2] += w * f;
      }
#pragma unroll
      for (int al = 0; al < 4; ++al) fs[al * NT + k] = (TA)(f * Si[al * NT + k]);
    }
  }
  // block totals of the three terms: only the warps that hold pairs (k < m)
  // reduce; the others hold zeros and skip the FP64 shuffle additions (the
  // totals are those of a reduction over every warp); the barriers also
  // publish fs
  {
    const int nwp = (m + 31) >> 5;
    if (warp < nwp) {
#pragma unroll
      for (int q = 0; q < 3; ++q) v[q] = tbk::warp_sum(v[q]);
    }
    if (lane == 0) {
#pragma unroll
      for (int q = 0; q < 3; ++q) red[warp * 3 + q] = warp < nwp ? v[q] : 0.0;
    }
    __syncthreads();
    if (threadIdx.x < 3) {
      double t = 0.0;
      for (int w = 0; w < nwp; ++w) t += red[w * 3 + threadIdx.x];
      tot[threadIdx.x] = t;
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    a.per_target[5 * i + 0] = 2.0 * tot[0];
    a.per_target[5 * i + 1] = 2.0 * a.kT * tot[1];
    a.per_target[5 * i + 2] = 2.0 * tot[2];
  }
  const int deg = a.h_off[i + 1] - a.h_off[i];
  const size_t base = (size_t)(i + a.h_off[i]);
  for (int blk = warp; blk <= deg; blk += RT / 32) {
    const double* pr = a.P + (base + blk) * 4 * NT;
    TA acc[16];
#pragma unroll
    for (int q = 0; q < 16; ++q) acc[q] = (TA)0;
    for (int k = lane; k < m; k += 32) {
      TA pb[4], sa[4];
#pragma unroll
      for (int be = 0; be < 4; ++be) {
        if constexpr (sizeof(TA) == 4) pb[be] = tbconv::d2f(pr[be * NT + k]);   // off the FP64 pipe
        else pb[be] = pr[be * NT + k];
      }
#pragma unroll
      for (int al = 0; al < 4; ++al) sa[al] = fs[al * NT + k];
#pragma unroll
      for (int be = 0; be < 4; ++be)
#pragma unroll
        for (int al = 0; al < 4; ++al) acc[be * 4 + al] += pb[be] * sa[al];
    }
    const TA t = tbk::warp_reduce16(acc, lane);   // lanes 2q hold entry q = be*4 + al
    if ((lane & 1) == 0) {
      if constexpr (sizeof(TA) == 4) a.rho[(base + blk) * 16 + (lane >> 1)] = tbconv::f2d(t);
      else a.rho[(base + blk) * 16 + (lane >> 1)] = (double)t;
    }
  }
}

// ---------------------------------------------------------------- forces

struct ForceArgs {
  int n;
  const double* pos;
  double L;
  const int* h_off;
  const int* h_idx;
  const double* dH;
  const double* rho;
  tb_gsp rep;
  double* bondf;
  double* F;
  double* per_target;   // n x 5, then the energy partials of force_sum_kernel's blocks
  int* st;
  double* energies;     // force_sum_kernel: the evaluation's energies (null: not formed)
  const double* mu;
  unsigned* ecnt;       // blocks done (zero between calls: the last block resets it)
};

// One thread per directed bond k -> j: the bond's Hellmann-Feynman term
// 2 sum_ab [rho^(k)_{j b,k a} + rho^(j)_{k a,j b}] dH_ab plus the pair
// repulsion, stored per bond; force_sum_kernel adds each atom's bonds in order.
// Runs of 32 consecutive bonds (one warp) are dealt out to the warps of all
// blocks in turn, so that every SM gets a share of this FP64-bound work in
// full warps.
__global__ void __launch_bounds__(64) force_bond_kernel(const ForceArgs a) {
  const int nb = a.h_off[a.n];
  const int wg = blockIdx.x + gridDim.x * (threadIdx.x >> 5);
  const int stride = gridDim.x * blockDim.x;
  for (int p = wg * 32 + (threadIdx.x & 31); p < nb; p += stride) {
  int lo = 0, hi = a.n;                 // source atom k: h_off[k] <= p < h_off[k+1]
  while (hi - lo > 1) {
    const int mid = (lo + hi) >> 1;
    if (a.h_off[mid] <= p) lo = mid; else hi = mid;
  }
  const int k = lo;
  const int j = a.h_idx[p];
  double* out = a.bondf + (size_t)p * 4;
  int l2 = a.h_off[j], h2 = a.h_off[j + 1];    // position of k in j's list
  while (l2 < h2) {
    const int mid = (l2 + h2) >> 1;
    if (a.h_idx[mid] < k) l2 = mid + 1; else h2 = mid;
  }
  if (l2 >= a.h_off[j + 1] || a.h_idx[l2] != k) {
    tbk::set_status(a.st, TB_ERR_INVALID_ARG, k);
    out[0] = out[1] = out[2] = out[3] = 0.0;
    continue;
  }
  const int q = p - a.h_off[k];
  const int rq = l2 - a.h_off[j];
  const double* rk = a.rho + ((size_t)(k + a.h_off[k]) + 1 + q) * 16;    // rho^(k)_{j b, k a} [b][a]
  const double* rj = a.rho + ((size_t)(j + a.h_off[j]) + 1 + rq) * 16;   // rho^(j)_{k a, j b} [a][b]
  const double* G = a.dH + (size_t)p * 48;
  double acc[3] = {0.0, 0.0, 0.0};
#pragma unroll
  for (int al = 0; al < 4; ++al)
#pragma unroll
    for (int be = 0; be < 4; ++be) {
      const double rs = rk[be * 4 + al] + rj[al * 4 + be];
#pragma unroll
      for (int kk = 0; kk < 3; ++kk) acc[kk] += rs * G[kk * 16 + al * 4 + be];
    }
  const double hL = 0.5 * a.L;
  double d[3];
#pragma unroll
  for (int kk = 0; kk < 3; ++kk) {
    const double x = a.pos[3 * j + kk] - a.pos[3 * k + kk];
    d[kk] = x > hL ? x - a.L : (x < -hL ? x + a.L : x);
  }
  const double r = sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
  double phi, dphi;
  tb_gsp_eval(a.rep, r, phi, dphi);
  const double sc = dphi / r;
  out[0] = 2.0 * acc[0] + sc * d[0];
  out[1] = 2.0 * acc[1] + sc * d[1];
  out[2] = 2.0 * acc[2] + sc * d[2];
  out[3] = 0.5 * phi;
  }
}

// Per atom: the force and repulsive energy as the sum of its bonds' terms in
// list order.  Then the energies: every block sums its atoms' E_band, -TS, N_e
// and E_rep (warp shuffles, then the two warps in order), writes the partial,
// and the last block to finish (a fence, then an atomic count) adds the
// partials in block order, a fixed order whatever the block schedule.
constexpr int FS_T = 64;
__global__ void __launch_bounds__(FS_T) force_sum_kernel(const ForceArgs a) {
  __shared__ double red[FS_T / 32 * 4];
  __shared__ int last;
  const int k = blockIdx.x * blockDim.x + threadIdx.x;
  const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
  double e[4] = {0.0, 0.0, 0.0, 0.0};
  if (k < a.n) {
    double f[4] = {0.0, 0.0, 0.0, 0.0};
    for (int p = a.h_off[k]; p < a.h_off[k + 1]; ++p)
#pragma unroll
      for (int c = 0; c < 4; ++c) f[c] += a.bondf[(size_t)p * 4 + c];
    a.F[3 * k] = f[0];
    a.F[3 * k + 1] = f[1];
    a.F[3 * k + 2] = f[2];
    a.per_target[5 * k + 3] = f[3];
    if (!(isfinite(f[0]) && isfinite(f[1]) && isfinite(f[2]))) tbk::set_status(a.st, TB_ERR_NONFINITE, k);
    e[0] = a.per_target[5 * k];
    e[1] = a.per_target[5 * k + 1];
    e[2] = a.per_target[5 * k + 2];
    e[3] = f[3];
  }
  if (!a.energies) return;                           // uniform over the grid
#pragma unroll
  for (int q = 0; q < 4; ++q) e[q] = tbk::warp_sum(e[q]);
  if (lane == 0) {
#pragma unroll
    for (int q = 0; q < 4; ++q) red[warp * 4 + q] = e[q];
  }
  __syncthreads();
  double* const part = a.per_target + (size_t)5 * a.n;
  if (threadIdx.x < 4) part[(size_t)blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x] + red[4 + threadIdx.x];
  __threadfence();
  __syncthreads();
  if (threadIdx.x == 0) last = atomicAdd(a.ecnt, 1u) == gridDim.x - 1;
  __syncthreads();
  if (!last) return;
  __threadfence();
  if (threadIdx.x < 4) {
    double t = 0.0;
    for (int b = 0; b < (int)gridDim.x; ++b) t += __ldcg(part + (size_t)b * 4 + threadIdx.x);
    red[threadIdx.x] = t;
  }
  __syncthreads();
  if (threadIdx.x == 0) {
    const double eb = red[0], ts = red[1], ne = red[2], er = red[3];
    a.energies[0] = eb;
    a.energies[1] = ts;
    a.energies[2] = eb + ts;
    a.energies[3] = er;
    a.energies[4] = eb + ts + er;
    a.energies[5] = ne;
    a.energies[6] = *a.mu;
    a.energies[7] = 0.0;
    *a.ecnt = 0u;
  }
}

// Virial of the pair-decomposed forces, W_ab = -1/2 sum over directed bonds of
// d_a f_b (d = R_j - R_k by minimum image, f the bond's force on k stored by
// force_bond_kernel), and the static pressure tr W / (3 L^3).  One block,
// atoms strided over the threads, fixed-order block reduction.
__global__ void __launch_bounds__(1024)
virial_kernel(int n, const double* pos, double L, const int* h_off, const int* h_idx,
              const double* bondf, double* W, double* pressure) {
  __shared__ double red[32 * 16];
  __shared__ double tot[16];
  double v[9] = {0, 0, 0, 0, 0, 0, 0, 0, 0};
  const double hL = 0.5 * L;
  for (int k = threadIdx.x; k < n; k += 1024) {
    for (int p = h_off[k]; p < h_off[k + 1]; ++p) {
      const int j = h_idx[p];
      double d[3];
#pragma unroll
      for (int c = 0; c < 3; ++c) {
        const double x = pos[3 * j + c] - pos[3 * k + c];
        d[c] = x > hL ? x - L : (x < -hL ? x + L : x);
      }
      const double* f = bondf + (size_t)p * 4;
#pragma unroll
      for (int a = 0; a < 3; ++a)
#pragma unroll
        for (int b = 0; b < 3; ++b) v[a * 3 + b] += d[a] * f[b];
    }
  }
  tbk::block_sum16<double, 9>(v, red, tot);
  if (threadIdx.x < 9) W[threadIdx.x] = -0.5 * tot[threadIdx.x];
  if (threadIdx.x == 0 && pressure)
    *pressure = -0.5 * (tot[0] + tot[4] + tot[8]) / (3.0 * L * L * L);
}

// energies[8] = {E_band, -TS, A, E_rep, E_tot, N(mu), mu, KE}; columns of
// per_target: E_band, -TS, N_e, E_rep, KE.  `cols` selects what to refresh.
__global__ void __launch_bounds__(ER_T)
energy_reduce_kernel(int n, const double* per_target, const double* mu, double* energies,
                     int with_ke) {
  __shared__ double red[32 * 5];
  __shared__ double tot[5];
  double v[5] = {0, 0, 0, 0, 0};
  // four rows' loads in flight per thread before their additions (in row order)
  for (int i0 = threadIdx.x; i0 < n; i0 += 4 * ER_T) {
    double x[4][5];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int i = i0 + u * ER_T;
#pragma unroll
      for (int c = 0; c < 5; ++c) x[u][c] = i < n ? per_target[5 * i + c] : 0.0;
    }
#pragma unroll
    for (int u = 0; u < 4; ++u)
#pragma unroll
      for (int c = 0; c < 5; ++c) v[c] += x[u][c];
  }
  tbk::block_sum<double, 5>(v, red, tot);
  if (threadIdx.x == 0) {
    if (with_ke) {
      energies[7] = tot[4];
    } else {
      energies[0] = tot[0];
      energies[1] = tot[1];
      energies[2] = tot[0] + tot[1];
      energies[3] = tot[3];
      energies[4] = tot[0] + tot[1] + tot[3];
      energies[5] = tot[2];
      energies[6] = *mu;
      energies[7] = 0.0;
    }
  }
}

// ---------------------------------------------------------------- Verlet

constexpr double ACC_CONV = 9.648533e-3;   // (eV/A/amu) -> A/fs^2

__global__ void kick_drift_kernel(int n, double* pos, double* vel, const double* F, double L,
                                  double dt, double mass) {
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const double v = vel[t] + 0.5 * dt * ACC_CONV / mass * F[t];
  vel[t] = v;
  double x = fmod(pos[t] + dt * v, L);
  if (x < 0.0) x += L;
  if (x >= L) x = 0.0;
  pos[t] = x;
}

__global__ void kick_kernel(int n, double* vel, const double* F, double dt, double mass,
                            double* per_target) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  double ke = 0.0;
  for (int kk = 0; kk < 3; ++kk) {
    const double v = vel[3 * i + kk] + 0.5 * dt * ACC_CONV / mass * F[3 * i + kk];
    vel[3 * i + kk] = v;
    ke += v * v;
  }
  per_target[5 * i + 4] = 0.5 * mass * ke / ACC_CONV;
}

// Weak-coupling (Berendsen) NPT scaling after one Verlet step.  Every
// block derives the two factors from the step's kinetic energy and virial (ten
// loads, identical arithmetic in every block); block 0 publishes the new box
// and the state.  A factor that is not a positive finite number leaves the
// system unchanged: a NaN or infinite factor (from a non-finite kinetic energy
// or virial) reports TB_ERR_NONFINITE, a finite but non-positive one (a target
// far from the current state for the coupling constants) TB_ERR_INVALID_ARG
// with info 0 for the thermostat's lambda^2, 1 for the barostat's mu^3.
__global__ void npt_scale_kernel(int n, double* pos, double* vel, double L, const double* W,
                                 const double* energies, double T0, double P0, double dt,
                                 double tau_T, double tau_P, double beta, double* L_new,
                                 double* state, int* st) {
  __shared__ double fac[2];
  if (threadIdx.x == 0) {
    const double KB = 8.617333262e-5;              // eV/K
    const double ke = energies[7];
    const double dof = n > 1 ? 3.0 * n - 3.0 : 3.0;
    const double T = 2.0 * ke / (KB * dof);
    const double V = L * L * L;
    const double P = (W[0] + W[4] + W[8] + 2.0 * ke) / (3.0 * V);
    // no kinetic temperature (all velocities zero): nothing to rescale
    const double lam2 = T > 0.0 ? 1.0 + dt / tau_T * (T0 / T - 1.0) : 1.0;
    const double mu3 = 1.0 - beta * dt / tau_P * (P0 - P);
    const bool fin = isfinite(lam2) && isfinite(mu3);
    const bool ok = fin && lam2 > 0.0 && mu3 > 0.0;
    fac[0] = ok ? sqrt(lam2) : 1.0;
    fac[1] = ok ? cbrt(mu3) : 1.0;
    if (blockIdx.x == 0) {
      *L_new = fac[1] * L;
      state[0] = T;
      state[1] = P;
      state[2] = fac[0];
      state[3] = fac[1];
      if (!fin) tbk::set_status(st, TB_ERR_NONFINITE, isfinite(lam2) ? 1 : 0);
      else if (!ok) tbk::set_status(st, TB_ERR_INVALID_ARG, lam2 > 0.0 ? 1 : 0);
    }
  }
  __syncthreads();
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= 3 * n) return;
  const double Ln = fac[1] * L;
  vel[t] *= fac[0];
  double x = fac[1] * pos[t];
  if (x >= Ln) x -= Ln;                             // mu x < mu L up to rounding
  if (x < 0.0) x = 0.0;
  pos[t] = x;
}

}  // namespace

tb_status launch_npt_berendsen(tb_ctx* c, int n, double* pos, double* vel, double L,
                               const double* W, const double* energies, double T0, double P0,
                               double dt, double tau_T, double tau_P, double beta,
                               double* L_new, double* state, cudaStream_t s) {
  const int grid = (3 * n + 255) / 256;
  npt_scale_kernel<<<grid > 0 ? grid : 1, 256, 0, s>>>(n, pos, vel, L, W, energies, T0, P0, dt,
                                                      tau_T, tau_P, beta, L_new, state,
                                                      c->d_status);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}

tb_status mu_configure(tb_ctx* c) {
  int dev = 0, max_smem = 0;
  TB_CUDA_TRY(cudaGetDevice(&dev));
  TB_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  c->mu_smem_max = max_smem - 8 * 1024;       // leave room for the static arrays
  TB_CUDA_TRY(cudaFuncSetAttribute(mu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                   c->mu_smem_max));
  int occ = 0;
  TB_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, mu_kernel, MT, c->mu_smem_max));
  if (occ < 1) return TB_ERR_CUDA;
  c->mu_grid = c->num_sms;   // one block per SM: co-resident, short final sums
  return TB_OK;
}

tb_status launch_mu(tb_ctx* c, int n, const double* lambda, const double* S,
                    double n_electrons, const double* mu_guess, double* mu,
                    double* n_count, cudaStream_t s) {
  return launch_mu_nt(c, n, 4 * c->p.r, lambda, S, n_electrons, mu_guess, mu, n_count, s);
}

tb_status launch_virial(tb_ctx* c, int n, const double* pos, double L, const int* h_off,
                        const int* h_idx, double* W, double* pressure, cudaStream_t s) {
  virial_kernel<<<1, 1024, 0, s>>>(n, pos, L, h_off, h_idx, c->bondf, W, pressure);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}

tb_status launch_energy_reduce(int n, const double* per_target, const double* mu,
                               double* energies, cudaStream_t s) {
  energy_reduce_kernel<<<1, ER_T, 0, s>>>(n, per_target, mu, energies, 0);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}

// mu search over records of NT pairs per target (NT = 4r for the Krylov record)
tb_status launch_mu_nt(tb_ctx* c, int n, int NT, const double* lambda, const double* S,
                       double n_electrons, const double* mu_guess, double* mu,
                       double* n_count, cudaStream_t s) {
  MuArgs a;
  a.npairs = (long long)n * NT;
  a.NT = NT;
  a.lambda = lambda;
  a.S = S;
  a.kT = c->p.kT;
  a.ikT = 1.0 / c->p.kT;
  a.ne = n_electrons;
  a.tolN = c->p.mu_tol * n_electrons;
  a.guess = mu_guess;
  a.mu_out = mu;
  a.ncount_out = n_count;
  a.iters_out = reinterpret_cast<int*>(c->mu_state);
  a.part = c->mu_part;
  a.bar = c->bar;
  a.max_iter = c->p.mu_max_iter;
  a.timeout = c->p.timeout_cycles;
  a.st = c->d_status;
  // one block per SM; each block stages its contiguous share of the pairs
  const int grid = c->mu_grid;
  a.per_block = (a.npairs + grid - 1) / grid;
  const size_t stage = (size_t)a.per_block * (sizeof(double2) + sizeof(float2) + sizeof(int));
  a.staged = stage <= (size_t)c->mu_smem_max ? 1 : 0;
  TB_CUDA_TRY(cudaMemsetAsync(c->bar, 0, sizeof(unsigned), s));
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(MT);
  cfg.dynamicSmemBytes = a.staged ? stage : 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TB_CUDA_TRY(cudaLaunchKernelEx(&cfg, mu_kernel, a));
  return TB_OK;
}

tb_status launch_forces(tb_ctx* c, int n, const double* pos, double L, const int* h_off,
                        const int* h_idx, const double* dHblk, const double* lambda,
                        const double* S, const double* P, const int* kdim, const double* mu,
                        double* F, double* energies, cudaStream_t s) {
  const int NT = 4 * c->p.r;
  RhoArgs ra{NT, h_off, kdim, lambda, S, P, mu, c->p.kT, 1.0 / c->p.kT, c->rho, c->per_target,
              c->d_status};
  if (c->p.prec != TB_PREC_FP64) rho_kernel<float><<<n, RT, 0, s>>>(ra);
  else rho_kernel<double><<<n, RT, 0, s>>>(ra);
  TB_CUDA_TRY(cudaGetLastError());
  ForceArgs fa{n, pos, L, h_off, h_idx, dHblk, c->rho, tb_repulsion_gsp(c->p), c->bondf, F,
               c->per_target, c->d_status, energies, mu, c->bar + 1};
  force_bond_kernel<<<16 * c->num_sms, 64, 0, s>>>(fa);
  TB_CUDA_TRY(cudaGetLastError());
  force_sum_kernel<<<(n + FS_T - 1) / FS_T, FS_T, 0, s>>>(fa);   // forces, then the energies
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}

tb_status launch_md_kick_drift(tb_ctx* c, int n, double* pos, double* vel, const double* F,
                               double L, double dt, double mass, cudaStream_t s) {
  kick_drift_kernel<<<(3 * n + 255) / 256, 256, 0, s>>>(n, pos, vel, F, L, dt, mass);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}

tb_status launch_md_kick(tb_ctx* c, int n, double* vel, const double* F, double dt,
                         double mass, double* energies, cudaStream_t s) {
  kick_kernel<<<(n + 255) / 256, 256, 0, s>>>(n, vel, F, dt, mass, c->per_target);
  TB_CUDA_TRY(cudaGetLastError());
  energy_reduce_kernel<<<1, ER_T, 0, s>>>(n, c->per_target, c->mu, energies, 1);
  TB_CUDA_TRY(cudaGetLastError());
  return TB_OK;
}

// ---------------------------------------------------------------------------
// Allocation-free variant of the chemical-potential search.
//
// Some callers cannot allocate device memory at all: code running inside a
// host runtime that owns every allocation (a pre-sized memory pool or arena,
// or a process where a cudaMalloc would synchronise the device at a bad
// moment).  They cannot create a tb_ctx either, because tb_ctx_create and
// tb_ctx_reserve allocate.  tb_find_mu_static gives them the mu search with
// its scratch (per-block partial sums and the grid-barrier counter) in this
// file-scope device array instead of in a context; the status words are the
// caller's.
//
// The array is sized for TB_FIND_MU_STATIC_MAX_BLOCKS blocks of the
// cooperative search (one block per SM); every GPU that loads the library
// holds it until the process exits.  All calls share it and it keeps the last
// call's contents, so the counter (and the caller's status words) are cleared
// on the stream before each launch; calls whose executions overlap on the GPU
// race on it.  The per-device set-up is guarded, so first calls from several
// host threads at once are safe.
namespace {

constexpr int kStaticPartDoubles = 2 * MU_PART * TB_FIND_MU_STATIC_MAX_BLOCKS;
// [0, kStaticPartDoubles) partial sums; then one 256-byte line whose first
// word is the grid-barrier counter (the rest of the line is unused)
static __device__ __align__(256) double g_mu_scratch[kStaticPartDoubles + 32];

struct StaticMuDevice {
  std::atomic<bool> ready{false};   // published with release after the fields below
  double* scratch = nullptr;   // device address of g_mu_scratch on this device
  int sms = 0;
  int smem_max = 0;
};
constexpr int kMaxDevices = 64;
StaticMuDevice g_static_mu[kMaxDevices];

// One-time set-up on the current device: device address of the scratch array
// (its name on the host is only a stand-in), SM count and the kernel's
// shared-memory limit.  Not capturable into a CUDA graph.
std::mutex g_static_mu_lock;

tb_status static_mu_setup(int dev) {
  StaticMuDevice& d = g_static_mu[dev];
  if (d.ready.load(std::memory_order_acquire)) return TB_OK;
  std::lock_guard<std::mutex> guard(g_static_mu_lock);
  if (d.ready.load(std::memory_order_relaxed)) return TB_OK;
  void* p = nullptr;
  if (cudaGetSymbolAddress(&p, g_mu_scratch) != cudaSuccess || !p) {
    cudaGetLastError();
    return TB_ERR_CUDA;
  }
  int sms = 0, max_smem = 0;
  TB_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  TB_CUDA_TRY(cudaDeviceGetAttribute(&max_smem, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev));
  const int smem = max_smem - 8 * 1024;
  TB_CUDA_TRY(cudaFuncSetAttribute(mu_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
  d.scratch = static_cast<double*>(p);
  d.sms = sms;
  d.smem_max = smem;
  d.ready.store(true, std::memory_order_release);
  return TB_OK;
}

}  // namespace

extern "C" tb_status tb_find_mu_static(int n, int r, const double* lambda, const double* S,
                                       double kT, double n_electrons, double mu_tol,
                                       int max_iter, const double* mu_guess, double* mu,
                                       double* n_count, int* status, void* stream) {
  if (n <= 0 || r < 1 || r > tbk::MAX_R || !lambda || !S || !mu || !status) return TB_ERR_INVALID_ARG;
  if (!(kT > 0.0) || !(n_electrons > 0.0) || !(mu_tol > 0.0) || max_iter < 1) return TB_ERR_INVALID_ARG;
  int dev = 0;
  TB_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kMaxDevices) return TB_ERR_INVALID_ARG;
  tb_status st = static_mu_setup(dev);
  if (st != TB_OK) return st;
  const StaticMuDevice& d = g_static_mu[dev];
  // one block per SM, as the context-based search; the array holds partials
  // for at most TB_FIND_MU_STATIC_MAX_BLOCKS blocks
  if (d.sms > TB_FIND_MU_STATIC_MAX_BLOCKS) return TB_ERR_CAPACITY;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const int NT = 4 * r;
  MuArgs a;
  a.npairs = (long long)n * NT;
  a.NT = NT;
  a.lambda = lambda;
  a.S = S;
  a.kT = kT;
  a.ikT = 1.0 / kT;
  a.ne = n_electrons;
  a.tolN = mu_tol * n_electrons;
  a.guess = mu_guess;
  a.mu_out = mu;
  a.ncount_out = n_count;
  a.iters_out = nullptr;
  a.part = d.scratch;
  unsigned* line = reinterpret_cast<unsigned*>(d.scratch + kStaticPartDoubles);
  a.bar = line;
  a.max_iter = max_iter;
  a.timeout = 4000000000LL;
  a.st = status;
  const int grid = d.sms;
  a.per_block = (a.npairs + grid - 1) / grid;
  const size_t stage = (size_t)a.per_block * (sizeof(double2) + sizeof(float2) + sizeof(int));
  a.staged = stage <= (size_t)d.smem_max ? 1 : 0;
  TB_CUDA_TRY(cudaMemsetAsync(line, 0, sizeof(unsigned), s));       // barrier counter
  TB_CUDA_TRY(cudaMemsetAsync(status, 0, 2 * sizeof(int), s));      // caller's status words
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(MT);
  cfg.dynamicSmemBytes = a.staged ? stage : 0;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  TB_CUDA_TRY(cudaLaunchKernelEx(&cfg, mu_kernel, a));
  return TB_OK;
}
