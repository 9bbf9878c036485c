// Cluster engine of the steady fixed point (Eqs. 13-21 with the convergence
// loop of Sec. V-C) for grids up to 256 x 256: one thread-block cluster per
// map, the map resident in shared memory for the whole solve.
#include <math.h>

#include "vs_fft.cuh"
#include "vs_solve_common.cuh"

using namespace vsfft;

namespace vsk {
namespace {

// Each map is held by one thread-block cluster for the whole solve, so it
// never leaves on-chip memory between iterations. CTA c of a cluster of n / 32 CTAs owns
//   - rows y in [32c, 32c + 32): 16 row FFTs, two rows packed per FFT;
//   - the x-frequency pairs (j, n - j), j in [16c, 16c + 16), pair 0 being
//     (0, n/2): 16 column FFTs, the two frequencies of a pair packed per FFT.
// Pairing k with n - k puts both operands of every DCT pre/post-twiddle in
// the CTA that produces them, so each exchange stores finished FFT inputs
// straight into the consumer's shared memory (st.shared::cluster) and one
// cluster barrier per exchange orders them. An iteration is: column phase
// (forward DCT along y, multiply by K / (1 - beta mu K) (Eq. 21 with
// alpha = 0), inverse DCT along y, push to the row owners), barrier, row
// phase (inverse DCT along x, the fused update of the streamed engine,
// forward DCT along x, push to the column owners together with the residual
// partials), barrier; then every CTA takes the same convergence decision from
// the same partials, so control flow stays uniform across the cluster. Global
// memory sees only the inputs (read) and theta (written). There are no spin
// waits: the cluster barriers are hardware barriers.

// Rows (and x-frequencies) a CTA owns at most; the cluster holds N / rows CTAs.
#ifndef VS_CL_ROWS
#define VS_CL_ROWS 32
#endif

template <int N>
struct ClShape {
  static constexpr int ROWS = N < VS_CL_ROWS ? N : VS_CL_ROWS;
  static constexpr int F = ROWS / 2;         // FFTs per CTA in each phase
  static constexpr int THREADS = 16 * F;     // one radix-16 butterfly per thread
  static constexpr int RANKS = N / ROWS;
  static constexpr int MIN_BLOCKS = THREADS <= 256 ? 2 : 1;
};

struct ClSlots {
  double part[kClMaxRanks];
  double part2[kClMaxRanks];
  float resid[kClMaxRanks];
  int flags[kClMaxRanks];
};

// Shared memory of one CTA for grid size N, in float2 units: row buffer
// [F][NP], column buffer [F][NP], spectral multiplier of the CTA's frequency
// pairs [N][F] (column index XOR-swizzled by the row), the first-pass FFT
// twiddles W_N^{j r} stored [r][j] (r < 16, j < N/16), the DCT twiddles
// W_4N^k (k < N), then the partials slots.
template <int N>
struct ClLayout {
  static constexpr int F = ClShape<N>::F;
  static constexpr int NP = N + N / 16 + 1;
  static constexpr int kBcol = F * NP;
  static constexpr int kLs = 2 * F * NP;
  static constexpr int kTwp = kLs + N * F;
  static constexpr int kTdct = kTwp + N;
  static constexpr int kSlots = kTdct + N;
  static constexpr size_t kBytes = (size_t)kSlots * sizeof(float2) + sizeof(ClSlots);
};

__device__ __forceinline__ unsigned cl_rank() {
  unsigned r;
  asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
  return r;
}
__device__ __forceinline__ unsigned cl_index() {
  unsigned r;
  asm volatile("mov.u32 %0, %%clusterid.x;" : "=r"(r));
  return r;
}
__device__ __forceinline__ void cl_arrive_relaxed() {
  asm volatile("barrier.cluster.arrive.relaxed.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_arrive_release() {
  asm volatile("barrier.cluster.arrive.release.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_wait() {
  asm volatile("barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ void cl_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// Address of the same shared-memory location in the CTA of cluster rank `rank`.
__device__ __forceinline__ unsigned cl_map(const void* p, unsigned rank) {
  unsigned a = (unsigned)__cvta_generic_to_shared(p), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void cl_put(unsigned a, float2 v) {
  asm volatile("st.shared::cluster.v2.f32 [%0], {%1, %2};" ::"r"(a), "f"(v.x), "f"(v.y) : "memory");
}
__device__ __forceinline__ void cl_put(unsigned a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void cl_put(unsigned a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void cl_put(unsigned a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}

// Digit-reversed position of frequency k in the output of the radix-16 x
// (N/16) forward FFT below (the same order as the streamed engine's tables).
template <int N>
__device__ __forceinline__ int cl_dr(int k) {
  return (k & 15) * (N / 16) + (k >> 4);
}

// Thread roles of the transforms (16 FFTs of length N = 16 R2 per buffer):
//   radix-16 role (the first 16 M1 threads, M1 = N/16): FFT f = t / M1 and
//     its positions j + M1 r, r < 16, j = t % M1;
//   radix-R2 role (all 256 threads): FFT f = t / 16 and its positions
//     16 b + r... stored as b R2 + r, r < R2, b = t % 16 (after the forward
//     pass these hold the frequencies k = 16 r + b).
// Forward transform = radix-16 pass (decimation in frequency, twiddled by
// W_N^{j r}) then radix-R2 pass; the inverse undoes them in reverse order.
// The radix-16 role keeps its 16 values in registers between the inverse and
// the forward transform along x, so the fixed-point update runs on them
// in place; the frequency k and its mirror N - k sit in lanes b and 16 - b of
// one half-warp and are paired with shuffles.
// BATCH: positions of the update whose inputs (P_leak0, P_dyn, s, theta of
// two rows) a thread loads together before using them, 1, 2 or 4: the depth of
// the global-load pipelining, a launch shape the plan's autotuner picks.
// Compensated FP32 accumulation (Knuth's two-sum): hi + lo carries the sum.
__device__ __forceinline__ void two_sum_add(float& hi, float& lo, float x) {
  const float tsum = hi + x, bp = tsum - hi;
  lo += (hi - (tsum - bp)) + (x - bp);
  hi = tsum;
}

// The physics variants (PHYS): the leakage factor g(theta) of a piecewise-linear
// table (Sec. II-E) and the field-point map of kappa(T) through the Kirchhoff
// transform (Eq. 10), as in the streamed engine's variant update.
__device__ __forceinline__ float cl_leak(const ClusterDev& P, float th) {
  if (P.leak_n == 0) return fmaf(P.beta, th, 1.f);
  int i = 0;
  while (i < P.leak_n - 2 && th >= P.leak_x[i + 1]) ++i;
  const float x0 = P.leak_x[i], y0 = P.leak_y[i];
  return fmaf((P.leak_y[i + 1] - y0) / (P.leak_x[i + 1] - x0), th - x0, y0);
}
__device__ __forceinline__ float cl_field_theta(const ClusterDev& P, float sk, float uu, int& flags) {
  if (P.cond == VS_COND_KIRCHHOFF) {
    float x = P.one_me * sk * uu / P.t_amb;
    if (!(x > -0.95f)) {
      flags |= kFlagRunaway;
      x = -0.95f;                         // keep theta finite; the map stops on the flag
    }
    return P.t_amb * expm1f(log1pf(x) / P.one_me);
  }
  const float den = fmaf(-P.alpha * sk, uu, 1.f);
  if (!(den > 0.05f)) flags |= kFlagRunaway;
  return sk * uu / den;
}
// dg/dtheta of the leakage factor at theta, and dtheta/du of the field map at u
// (s = 1): the uniform start's preconditioner for the variants.
__device__ __forceinline__ float cl_leak_slope(const ClusterDev& P, float th) {
  if (P.leak_n == 0) return P.beta;
  int i = 0;
  while (i < P.leak_n - 2 && th >= P.leak_x[i + 1]) ++i;
  return (P.leak_y[i + 1] - P.leak_y[i]) / (P.leak_x[i + 1] - P.leak_x[i]);
}
__device__ __forceinline__ float cl_field_dtheta(const ClusterDev& P, float u) {
  if (P.cond == VS_COND_KIRCHHOFF)
    return expf(log1pf(P.one_me * u / P.t_amb) * (1.f / P.one_me - 1.f));
  const float den = fmaf(-P.alpha, u, 1.f);
  return 1.f / (den * den);
}
__device__ __forceinline__ float cl_field_u(const ClusterDev& P, float sk, float t0) {
  if (P.cond == VS_COND_KIRCHHOFF)
    return P.t_amb * expm1f(P.one_me * log1pf(t0 / P.t_amb)) / (P.one_me * sk);
  return t0 / (sk * fmaf(P.alpha, t0, 1.f));
}

// CF: the one-shot closed form (Sec. IV-C, Eqs. 21, 25, 26) instead of the
// fixed point, on the same cluster layout (see the closed-form block below).
// PHYS: the physics variants in the update (P.beta is then the preconditioner
// slope, the table's at theta = 0); a cold map starts from the die's uniform
// mode of the variant (below).
template <int N, int BATCH, bool CF = false, bool PHYS = false>
__global__ void __launch_bounds__(ClShape<N>::THREADS, ClShape<N>::MIN_BLOCKS)
    k_solve_cluster(ClusterDev P) {
  constexpr int kClBatch = BATCH;
  using Lay = ClLayout<N>;
  constexpr int kClRows = ClShape<N>::ROWS, kClF = ClShape<N>::F;
  constexpr int kClThreads = ClShape<N>::THREADS, ranks = ClShape<N>::RANKS;
  constexpr int NP = Lay::NP, half = N / 2;
  constexpr int M1 = N / 16, R2 = N / 16;
  constexpr int kP16 = kClF * M1;
  extern __shared__ __align__(16) float2 cl_smem[];
  __shared__ double red_d[kClThreads / 32];
  __shared__ float red_f[kClThreads / 32];
  __shared__ int red_i[kClThreads / 32];
  const unsigned rank = cl_rank();
  const int b = __ldg(&P.order[cl_index()]);
  const MapDesc& d = P.maps[b];   // fields are read where used
  float2* brow = cl_smem;
  float2* bcol = cl_smem + Lay::kBcol;
  float2* Ls = cl_smem + Lay::kLs;
  float2* twp = cl_smem + Lay::kTwp;
  float2* tw = cl_smem + Lay::kTdct;
  ClSlots* slots = reinterpret_cast<ClSlots*>(cl_smem + Lay::kSlots);
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  // radix-16 role of the row phase: lanes run along x (coalesced inputs);
  // the mirror position N - 1 - m sits in lane M1 - 1 - j16 of the group
  const bool p16 = t < kP16;
  const int f16 = t / M1, j16 = t % M1;
  const int partner16 = (lane & ~(M1 - 1)) | (M1 - 1 - j16);
  // radix-R2 role: warp w holds the frequency digits blk = w and 16 - w
  // (w = 0: 0 and 8) for all 16 FFTs, one FFT per lane of each half-warp, so
  // frequency k and N - k are in lanes l and l ^ 16 and the stores to a peer
  // run along the FFTs (consecutive rows or pairs) in every half-warp
  const int f2 = lane & 15;
  const int blk = lane < 16 ? warp : (warp == 0 ? 8 : 16 - warp);
  const int partner2 = (blk == 0 || blk == 8) ? lane : (lane ^ 16);
  // radix-16 role of the column phase: warp w < M1/2 holds positions j = w
  // and M1 - 1 - w for all 16 frequency pairs (lanes), so the two rows of a
  // row pair are in lanes l and l ^ 16 and the stores run along the pairs
  const bool c16 = warp < M1 / 2;
  const int jc = lane & 15;
  const int j16c = lane < 16 ? warp : M1 - 1 - warp;
  const int y0 = (int)rank * kClRows;
  const int j0 = (int)rank * kClF;
  const float beta = P.beta, alpha = P.alpha;
  for (int i = t; i < N; i += kClThreads) {
    const int r = i / M1, j = i % M1;
    twp[i] = __ldg(&d.tw4n[4 * j * r]);
    tw[i] = __ldg(&d.tw4n[i]);
  }
  __syncthreads();

  auto load16 = [&](const float2* buf, float2* v, int f, int j) {
#pragma unroll
    for (int r = 0; r < 16; ++r) v[r] = buf[f * NP + pad(j + r * M1)];
  };
  auto store16 = [&](float2* buf, const float2* v, int f, int j) {
#pragma unroll
    for (int r = 0; r < 16; ++r) buf[f * NP + pad(j + r * M1)] = v[r];
  };
  auto base2 = [&](float2* buf) { return buf + f2 * NP + blk * R2 + ((blk * R2) >> 4); };
  auto fwd16 = [&](float2* v, int j) {
    dft16<true>(v);
    if (M1 > 1) {
#pragma unroll
      for (int r = 1; r < 16; ++r) v[r] = cmul(v[r], twp[r * M1 + j]);
    }
  };
  auto inv16 = [&](float2* v, int j) {
    if (M1 > 1) {
#pragma unroll
      for (int r = 1; r < 16; ++r) v[r] = cmulc(v[r], twp[r * M1 + j]);
    }
    dft16<false>(v);
  };
  auto shfl2 = [&](float2 v, int src) {
    return make_float2(__shfl_sync(0xffffffffu, v.x, src), __shfl_sync(0xffffffffu, v.y, src));
  };

  int status = VS_OK, iters = 0, growth = 0;
  float prev = INFINITY;
  double mu = 0.0;
  bool stop = false;
  // the residual and flags of an iterate to every CTA of the cluster
  auto put_slots = [&]() {
    if (t == 0) {
      float rm = 0.f;
      int fo = 0;
      for (int w = 0; w < kClThreads / 32; ++w) {
        rm = fmaxf(rm, red_f[w]);
        fo |= red_i[w];
      }
      for (int r = 0; r < ranks; ++r) {
        cl_put(cl_map(&slots->resid[rank], (unsigned)r), rm);
        cl_put(cl_map(&slots->flags[rank], (unsigned)r), fo);
      }
    }
  };
  // the convergence decision of iterate `it` from the residuals and flags in
  // the slots, the same in every thread of every CTA of the cluster
  auto decide = [&](int it) {
    float rr = 0.f;
    int ff = 0;
    for (int r = 0; r < ranks; ++r) {
      rr = fmaxf(rr, slots->resid[r]);
      ff |= slots->flags[r];
    }
    iters = it;
    if (ff & kFlagNonfinite) {
      status = VS_ERR_NONFINITE;
      stop = true;
    } else if (ff & kFlagRunaway) {
      status = VS_ERR_RUNAWAY;
      stop = true;
    } else if (converged(rr, prev, it, P.tol, P.stop_rule)) {
      status = VS_OK;
      stop = true;
    } else {
      growth = (it > 2 && rr > prev) ? growth + 1 : 0;
      if (it >= P.max_iter || growth >= 5) {
        status = VS_ERR_NO_CONVERGENCE;
        stop = true;
      }
    }
    prev = rr;
  };

  // closed form: the sums of P_leak0 and P_dyn over this CTA's cells, taken in
  // the first-source row pass (the closed form has no separate means pass)
  float cf_lh = 0.f, cf_ll = 0.f, cf_dh = 0.f, cf_dl = 0.f;

  // Row phase. mode 1: initial source from theta_0, the warm start's map or
  // the uniform th0 (not stored); 2: iteration (brow holds the spectra of the
  // column phase, pre-twiddled, at digit-reversed places); 3: the first
  // iteration after a uniform theta_0 = th0 (not read). mu is the mean leakage
  // of the preconditioner (source term - beta mu u). early > 0: iterate
  // `early` decides before the forward transform along x (the residuals are
  // exchanged on a cluster barrier whose wait overlaps the radix-16 pass in
  // registers), so a stopping map skips the transform's shared-memory pass
  // and the stores into the column owners; a map that goes on then needs a
  // cluster barrier before the next column phase, as with early = 0.
  auto row_phase = [&](int mode, float mu, float th0, float& resid, int& flags, int early) {
    const bool iter = mode >= 2;
    if (iter) {
      // brow holds the spectra in natural frequency order: the radix-R2 pass
      // takes frequencies blk + 16 r and leaves its outputs in place
      float2* p = brow + f2 * NP;
      float2 w[R2];
#pragma unroll
      for (int r = 0; r < R2; ++r) w[r] = p[pad(blk + 16 * r)];
      dftR<R2, false>(w);
#pragma unroll
      for (int r = 0; r < R2; ++r) p[pad(blk + 16 * r)] = w[r];
      __syncthreads();
    }
    float2 v[16];
    if (p16 && iter) {
      // radix-16 inputs of this thread: block j16 of the pass above
#pragma unroll
      for (int r = 0; r < 16; ++r) v[r] = brow[f16 * NP + pad(16 * j16 + r)];
    }
    if (iter) __syncthreads();   // the forward pass below rewrites brow in another order
    if (p16) {
      if (iter) inv16(v, j16);   // v[r] = u at Makhoul position j16 + M1 r of rows ya, ya + 1
      // Positions m (< N/2, x = 2m) of this lane and N - 1 - m (x + 1) of the
      // mirror lane are updated together, so every input is read as a
      // coalesced float2 (x, x + 1); u and q of x + 1 travel by shuffle.
      const size_t row_a = (size_t)(y0 + 2 * f16) * N;
      auto ld2 = [&](const float* p, size_t idx) {
        return __ldg(reinterpret_cast<const float2*>(p + idx));
      };
#pragma unroll
      for (int r0 = 0; r0 < 8; r0 += kClBatch) {
        float2 pl[kClBatch][2], pd[kClBatch][2], sk[kClBatch][2], old[kClBatch][2];
#pragma unroll
        for (int u = 0; u < kClBatch; ++u) {
          const int x = 2 * (j16 + (r0 + u) * M1);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const size_t idx = row_a + (size_t)h * N + x;
            pl[u][h] = ld2(d.p_leak0, idx);
            pd[u][h] = ld2(d.p_dyn, idx);
            if constexpr (CF) {
              two_sum_add(cf_lh, cf_ll, pl[u][h].x);
              two_sum_add(cf_lh, cf_ll, pl[u][h].y);
              two_sum_add(cf_dh, cf_dl, pd[u][h].x);
              two_sum_add(cf_dh, cf_dl, pd[u][h].y);
            }
            sk[u][h] = d.s ? ld2(d.s, idx) : make_float2(1.f, 1.f);
            old[u][h] = mode == 2 ? *reinterpret_cast<const float2*>(d.theta + idx)
                        : (mode == 1 && d.theta_init) ? ld2(d.theta_init, idx)
                        : make_float2(th0, th0);
          }
        }
#pragma unroll
        for (int u = 0; u < kClBatch; ++u) {
          const int r = r0 + u;
          const int x = 2 * (j16 + r * M1);
          const float2 um = shfl2(v[15 - r], partner16);   // u at x + 1 (mirror lane)
          float qe[2], qo[2];
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const size_t idx = row_a + (size_t)h * N + x;
            float th[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float PL = e ? pl[u][h].y : pl[u][h].x, PD = e ? pd[u][h].y : pd[u][h].x;
              const float S = e ? sk[u][h].y : sk[u][h].x, O = e ? old[u][h].y : old[u][h].x;
              float q;
              if constexpr (PHYS) {
                // P_dyn + P_leak0 g(theta) - b u, b = slope mu (Sec. IV-C)
                if (mode == 1) {
                  const float u0 = O == 0.f ? 0.f : cl_field_u(P, S, O);
                  th[e] = O;
                  q = fmaf(PL, cl_leak(P, O), PD) - beta * mu * u0;
                } else {
                  const float uu = e ? (h ? um.y : um.x) : (h ? v[r].y : v[r].x);
                  th[e] = cl_field_theta(P, S, uu, flags);
                  if (!isfinite(th[e])) flags |= kFlagNonfinite;
                  else resid = fmaxf(resid, fabsf(th[e] - O));
                  q = fmaf(PL, cl_leak(P, th[e]), PD) - beta * mu * uu;
                }
              } else if (mode == 1) {
                // u_0 = theta_0 / (s (1 + alpha theta_0))
                const float u0 = __fdividef(O, S * fmaf(alpha, O, 1.f));
                th[e] = O;
                q = PD + PL + beta * fmaf(PL, O, -mu * u0);
              } else {
                const float uu = e ? (h ? um.y : um.x) : (h ? v[r].y : v[r].x);
                const float den = fmaf(-alpha * S, uu, 1.f);
                if (!(den > 0.05f)) flags |= kFlagRunaway;
                th[e] = __fdividef(S * uu, den);   // 2 ulp, far below the FFT noise
                if (!isfinite(th[e])) flags |= kFlagNonfinite;
                else resid = fmaxf(resid, fabsf(th[e] - O));
                q = PD + PL + beta * fmaf(PL, th[e], -mu * uu);
              }
              (e ? qo : qe)[h] = q;
            }
            // theta_0 is kept only for a warm start (a uniform one is th0)
            if (mode == 2 || mode == 3 || d.theta_init)
              *reinterpret_cast<float2*>(d.theta + idx) = make_float2(th[0], th[1]);
          }
          v[r] = make_float2(qe[0], qe[1]);
          v[15 - r] = shfl2(make_float2(qo[0], qo[1]), partner16);
        }
      }
      if (!early) {
        fwd16(v, j16);
        store16(brow, v, f16, j16);
      }
    }
    // per-warp partials of the residual and flags of an iterate
    if (iter) {
#pragma unroll
      for (int o = 16; o > 0; o >>= 1) {
        resid = fmaxf(resid, __shfl_down_sync(0xffffffffu, resid, o));
        flags |= __shfl_down_sync(0xffffffffu, flags, o);
      }
    }
    if (lane == 0) {
      red_f[warp] = resid;
      red_i[warp] = flags;
    }
    __syncthreads();
    if (early) {
      put_slots();
      cl_arrive_release();
      if (p16) fwd16(v, j16);
      cl_wait();
      decide(early);
      if (stop) return;
      if (p16) store16(brow, v, f16, j16);
      __syncthreads();
    }
    // radix-R2 pass: Z[k], k = 16 r + blk; pair with N - k from the partner
    // lane, DCT-II post-twiddle, store into the column owner
    float2 z[R2];
    {
      const float2* p = base2(brow);
#pragma unroll
      for (int r = 0; r < R2; ++r) z[r] = p[r];
    }
    dftR<R2, true>(z);
    // lanes 0-15 of a half-warp hold 16 consecutive row pairs of one pair k:
    // each store below is one contiguous run in the owner's column buffer
    const unsigned oe = (unsigned)pad(y0 / 2 + f2) * 8u;
    const unsigned oo = (unsigned)pad(N - 1 - y0 / 2 - f2) * 8u;
#pragma unroll
    for (int r = 0; r < R2 / 2; ++r) {
      // what the partner needs at its index r: Z[N - k'] for its k' = 16 r + (16 - blk)
      const float2 give = blk == 0 ? z[r == 0 ? R2 / 2 : R2 - r] : z[R2 - 1 - r];
      const float2 zn = shfl2(give, partner2);
      const int k = 16 * r + blk;
      float2 ea, eb;
      if (k == 0) {
        const float2 x0 = dct_post(z[0], z[0], tw[0]), xh = dct_post(zn, zn, tw[half]);
        ea = make_float2(x0.x, xh.x);
        eb = make_float2(x0.y, xh.y);
      } else {
        const float2 xk = dct_post(z[r], zn, tw[k]), xn = dct_post(zn, z[r], tw[N - k]);
        ea = make_float2(xk.x, xn.x);
        eb = make_float2(xk.y, xn.y);
      }
      const unsigned dst = cl_map(bcol, (unsigned)r) + (unsigned)(blk * NP) * 8u;   // owner k / 16 = r
      cl_put(dst + oe, ea);
      cl_put(dst + oo, eb);
    }
  };

  // Column phase: bcol holds, for this CTA's frequency pairs, the x-spectra
  // of all rows at the Makhoul positions of y.
  auto col_phase = [&]() {
    if (c16) {
      float2 v[16];
      load16(bcol, v, jc, j16c);
      fwd16(v, j16c);
      store16(bcol, v, jc, j16c);
    }
    __syncthreads();
    {
      float2* p = base2(bcol);
      float2 z[R2], e[R2];
#pragma unroll
      for (int r = 0; r < R2; ++r) z[r] = p[r];
      dftR<R2, true>(z);
      const int jj = f2;
#pragma unroll
      for (int r = 0; r < R2; ++r) {
        const float2 give = blk == 0 ? z[(R2 - r) % R2] : z[R2 - 1 - r];
        const float2 zn = shfl2(give, partner2);   // Z[N - q]
        const int q = 16 * r + blk, qn = N - q;
        const float2 L = Ls[q * kClF + (jj ^ (q & (kClF - 1)))];
        float2 y = dct_post(z[r], zn, tw[q]);
        y.x *= L.x;
        y.y *= L.y;
        float2 yn;
        if (q == 0) {
          yn = make_float2(0.f, 0.f);
        } else if (q == half) {
          yn = y;
        } else {
          const float2 Ln = Ls[qn * kClF + (jj ^ (qn & (kClF - 1)))];
          yn = dct_post(zn, z[r], tw[qn]);
          yn.x *= Ln.x;
          yn.y *= Ln.y;
        }
        e[r] = dct_pre(y.x, yn.x, y.y, yn.y, tw[q]);
      }
      dftR<R2, false>(e);
#pragma unroll
      for (int r = 0; r < R2; ++r) p[r] = e[r];
    }
    __syncthreads();
    if (c16) {
      float2 v[16];
      load16(bcol, v, jc, j16c);
      inv16(v, j16c);   // v[r] = column data at Makhoul position j16c + M1 r of y
      const int j = j0 + jc;
      const int pa = j, pb = j == 0 ? half : N - j;
      const float2 twa = tw[pa], twb = tw[pb];
      const unsigned ra = (unsigned)pad(pa) * 8u, rb = (unsigned)pad(pb) * 8u;
      // the rows ya = 2 m (m = j16c + M1 r < N/2) and ya + 1 (position
      // N - 1 - m, lane ^ 16); lanes 0-15 hold 16 consecutive pairs, whose
      // values land on consecutive natural-order frequencies of the owner
#pragma unroll
      for (int r = 0; r < 8; ++r) {
        const float2 vb = shfl2(v[15 - r], lane ^ 16);
        const float2 va = v[r];
        float2 ea, eb;
        if (j == 0) {
          ea = dct_pre(va.x, 0.f, vb.x, 0.f, twa);
          eb = dct_pre(va.y, va.y, vb.y, vb.y, twb);
        } else {
          ea = dct_pre(va.x, va.y, vb.x, vb.y, twa);
          eb = dct_pre(va.y, va.x, vb.y, vb.x, twb);
        }
        const int ya = 2 * (j16c + r * M1);
        const unsigned dst = cl_map(brow, (unsigned)(ya / kClRows)) +
                             (unsigned)(((ya % kClRows) >> 1) * NP) * 8u;
        cl_put(dst + ra, ea);
        cl_put(dst + rb, eb);
      }
    }
  };

  auto cluster_mu = [&]() {
    double sum = 0.0;
    for (int r = 0; r < ranks; ++r) sum += slots->part[r];
    return sum / ((double)N * N);
  };

  // this CTA's kernel values for the multiplier table (pairs a / b of frequency
  // column j, N / 16 per thread), loaded while the cluster exchanges the
  // leakage partial sums
  constexpr int kKv = kClF * N / kClThreads;
  float2 kv[kKv];
  auto load_k = [&]() {
#pragma unroll
    for (int i = 0; i < kKv; ++i) {
      const int it = t + i * kClThreads;
      const int q = it % N, j = j0 + it / N;
      const int pa = j == 0 ? 0 : j, pb = j == 0 ? half : N - j;
      kv[i] = make_float2(__ldg(&d.Kt[(size_t)pa * N + q]), __ldg(&d.Kt[(size_t)pb * N + q]));
    }
  };
  cl_arrive_relaxed();  // peers store into this CTA only after every CTA started

  // The means of the inputs over the die: mu = mean(P_leak0) (Sec. IV-C) and,
  // for a cold start, mean(P_dyn), as compensated FP32 sums.
  const bool cold = !d.theta_init;
  if constexpr (!CF) {
    float lh = 0.f, ll = 0.f, dh = 0.f, dl = 0.f;
    auto add2 = [](float& hi, float& lo, float x) {
      const float tsum = hi + x, bp = tsum - hi;
      lo += (hi - (tsum - bp)) + (x - bp);
      hi = tsum;
    };
    // all loads of a thread are issued before the sums (first touch of the
    // inputs: HBM latency)
    constexpr int kM = kClRows * N / 4 / kClThreads;
    float4 a[kM], c[kM];
#pragma unroll
    for (int k = 0; k < kM; ++k) {
      const size_t idx = (size_t)y0 * N + 4 * (size_t)(t + k * kClThreads);
      a[k] = __ldg(reinterpret_cast<const float4*>(d.p_leak0 + idx));
      c[k] = cold ? __ldg(reinterpret_cast<const float4*>(d.p_dyn + idx)) : make_float4(0.f, 0.f, 0.f, 0.f);
    }
#pragma unroll
    for (int k = 0; k < kM; ++k) {
      add2(lh, ll, a[k].x);
      add2(lh, ll, a[k].y);
      add2(lh, ll, a[k].z);
      add2(lh, ll, a[k].w);
      add2(dh, dl, c[k].x);
      add2(dh, dl, c[k].y);
      add2(dh, dl, c[k].z);
      add2(dh, dl, c[k].w);
    }
    const double tot_l = block_sum((double)lh + (double)ll, red_d);
    const double tot_d = cold ? block_sum((double)dh + (double)dl, red_d) : 0.0;
    cl_wait();
    if (t == 0)
      for (int r = 0; r < ranks; ++r) {
        cl_put(cl_map(&slots->part[rank], (unsigned)r), tot_l);
        cl_put(cl_map(&slots->part2[rank], (unsigned)r), tot_d);
      }
    load_k();
    cl_sync();
    mu = cluster_mu();
  }
  if constexpr (CF) {
    // One-shot closed form of the map (the three-pass kernels of vs_closed.cu
    // compute the same):
    //   u = L_det * q + (P_leak0 - mu) . r,  q = P_dyn + P_leak0,  theta = phi(u)
    //   L_det = K / (1 - beta mu K) (Eq. 21), r = beta L_det^2 * q (Eq. 25 to
    //   first order) or beta L_det^2 * delta_centre sum(q) (Eq. 26).
    // Forward DCT of q along x (the first-source pass with theta_0 = 0), along
    // y, both multipliers; the random part's spectra wait in the multiplier
    // table's place while the L_det part goes back through the inverse
    // transforms into theta (as a staging copy of u_det); then the random
    // part follows and the last row pass combines the two. The means come
    // from the first row pass (q needs no mean), exchanged on its barrier.
    const bool impulse = P.cf_mode == VS_CF_IMPULSE;
    cl_wait();                                      // every CTA has started
    load_k();
    {
      float r0 = 0.f;
      int f0 = 0;
      row_phase(1, 0.f, 0.f, r0, f0, 0);          // q = P_dyn + P_leak0, forward along x
    }
    {
      const double tot_l = block_sum((double)cf_lh + (double)cf_ll, red_d);
      const double tot_d = block_sum((double)cf_dh + (double)cf_dl, red_d);
      if (t == 0)
        for (int r = 0; r < ranks; ++r) {
          cl_put(cl_map(&slots->part[rank], (unsigned)r), tot_l);
          cl_put(cl_map(&slots->part2[rank], (unsigned)r), tot_d);
        }
    }
    cl_sync();
    mu = cluster_mu();
    double tot_q = 0.0;
    for (int r = 0; r < ranks; ++r) tot_q += slots->part[r] + slots->part2[r];
    const float mu_f = (float)mu, nn = (float)N * (float)N;
    int cf_flags = ((double)beta * mu * (double)d.kmax >= 0.999) ? kFlagRunaway : 0;
    {
      const float bm = beta * mu_f;
      const float inv_n2 = 1.f / nn;
#pragma unroll
      for (int i = 0; i < kKv; ++i) {
        const int it = t + i * kClThreads;
        const int q = it % N, jj = it / N;
        const float ka = kv[i].x, kb = kv[i].y;
        Ls[q * kClF + (jj ^ (q & (kClF - 1)))] =
            make_float2(ka / (1.f - bm * ka) * inv_n2, kb / (1.f - bm * kb) * inv_n2);
      }
      __syncthreads();
    }
    // the radix-16 inverse along y of bcol and the stores into the row owners
    auto col_push = [&]() {
      __syncthreads();
      if (c16) {
        float2 v[16];
        load16(bcol, v, jc, j16c);
        inv16(v, j16c);
        const int j = j0 + jc;
        const int pa = j, pb = j == 0 ? half : N - j;
        const float2 twa = tw[pa], twb = tw[pb];
        const unsigned ra = (unsigned)pad(pa) * 8u, rb = (unsigned)pad(pb) * 8u;
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const float2 vb = shfl2(v[15 - r], lane ^ 16);
          const float2 va = v[r];
          float2 ea, eb;
          if (j == 0) {
            ea = dct_pre(va.x, 0.f, vb.x, 0.f, twa);
            eb = dct_pre(va.y, va.y, vb.y, vb.y, twb);
          } else {
            ea = dct_pre(va.x, va.y, vb.x, vb.y, twa);
            eb = dct_pre(va.y, va.x, vb.y, vb.x, twb);
          }
          const int ya = 2 * (j16c + r * M1);
          const unsigned dst = cl_map(brow, (unsigned)(ya / kClRows)) +
                               (unsigned)(((ya % kClRows) >> 1) * NP) * 8u;
          cl_put(dst + ra, ea);
          cl_put(dst + rb, eb);
        }
      }
    };
    // forward along y and both multipliers; the random part's pre-twiddled
    // spectra go to the multiplier table's place ([r][thread]), the L_det
    // part back to bcol
    {
      if (c16) {
        float2 v[16];
        load16(bcol, v, jc, j16c);
        fwd16(v, j16c);
        store16(bcol, v, jc, j16c);
      }
      __syncthreads();
      float2* p = base2(bcol);
      float2 z[R2], e1[R2], e2[R2];
#pragma unroll
      for (int r = 0; r < R2; ++r) z[r] = p[r];
      dftR<R2, true>(z);
      const int jj = f2, j = j0 + jj;
      const int pa = j == 0 ? 0 : j, pb = j == 0 ? half : N - j;
      // 2-D DCT-II of a unit impulse at the centre cell c = N/2:
      // cos(pi p (2c + 1) / 2N) cos(pi k (2c + 1) / 2N)
      auto dimp = [&](int f) { return cospif((float)((f * (N + 1)) % (4 * N)) / (float)(2 * N)); };
      const float da = dimp(pa), db = dimp(pb);
#pragma unroll
      for (int r = 0; r < R2; ++r) {
        const float2 give = blk == 0 ? z[(R2 - r) % R2] : z[R2 - 1 - r];
        const float2 zn = shfl2(give, partner2);   // Z[N - q]
        const int q = 16 * r + blk, qn = N - q;
        const float2 L = Ls[q * kClF + (jj ^ (q & (kClF - 1)))];
        const float2 y = dct_post(z[r], zn, tw[q]);
        // random-part multiplier beta L_det^2 / N^2 = beta L^2 N^2 (L holds L_det / N^2)
        auto rnd = [&](float2 x, float2 l, int qq) {
          const float dq = impulse ? dimp(qq) : 0.f;
          return make_float2((impulse ? da * dq : x.x) * beta * l.x * l.x * nn,
                             (impulse ? db * dq : x.y) * beta * l.y * l.y * nn);
        };
        float2 y1 = make_float2(y.x * L.x, y.y * L.y), y2 = rnd(y, L, q);
        float2 y1n, y2n;
        if (q == 0) {
          y1n = y2n = make_float2(0.f, 0.f);
        } else if (q == half) {
          y1n = y1;
          y2n = y2;
        } else {
          const float2 Ln = Ls[qn * kClF + (jj ^ (qn & (kClF - 1)))];
          const float2 yn = dct_post(zn, z[r], tw[qn]);
          y1n = make_float2(yn.x * Ln.x, yn.y * Ln.y);
          y2n = rnd(yn, Ln, qn);
        }
        e1[r] = dct_pre(y1.x, y1n.x, y1.y, y1n.y, tw[q]);
        e2[r] = dct_pre(y2.x, y2n.x, y2.y, y2n.y, tw[q]);
      }
      dftR<R2, false>(e1);
      dftR<R2, false>(e2);
      __syncthreads();                              // every thread is done with Ls
#pragma unroll
      for (int r = 0; r < R2; ++r) {
        p[r] = e1[r];
        Ls[r * kClThreads + t] = e2[r];
      }
    }
    col_push();                                     // L_det part -> the row owners
    cl_sync();
    // inverse along x of brow: v[r] = u at Makhoul position j16 + M1 r of rows
    // ya, ya + 1 (the radix-R2 pass first, as in the row phase)
    auto row_inverse = [&](float2* v) {
      {
        float2* p = brow + f2 * NP;
        float2 w[R2];
#pragma unroll
        for (int r = 0; r < R2; ++r) w[r] = p[pad(blk + 16 * r)];
        dftR<R2, false>(w);
#pragma unroll
        for (int r = 0; r < R2; ++r) p[pad(blk + 16 * r)] = w[r];
      }
      __syncthreads();
      if (p16) {
#pragma unroll
        for (int r = 0; r < 16; ++r) v[r] = brow[f16 * NP + pad(16 * j16 + r)];
      }
      __syncthreads();
      if (p16) inv16(v, j16);
    };
    const size_t row_a = (size_t)(y0 + 2 * f16) * N;
    {
      float2 v[16];
      row_inverse(v);
      if (p16) {
        // u_det of the cells (x, x + 1) of rows ya, ya + 1, staged in theta
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const float2 um = shfl2(v[15 - r], partner16);   // at x + 1 (mirror lane)
          const int x = 2 * (j16 + r * M1);
          *reinterpret_cast<float2*>(d.theta + row_a + x) = make_float2(v[r].x, um.x);
          *reinterpret_cast<float2*>(d.theta + row_a + N + x) = make_float2(v[r].y, um.y);
        }
      }
    }
    cl_sync();                                      // every CTA has read its brow
    {
      float2* p = base2(bcol);
#pragma unroll
      for (int r = 0; r < R2; ++r) p[r] = Ls[r * kClThreads + t];
    }
    col_push();                                     // random part -> the row owners
    cl_sync();
    {
      const float scale = impulse ? (float)tot_q : 1.f;
      float2 v[16];
      row_inverse(v);
      if (p16) {
#pragma unroll
        for (int r = 0; r < 8; ++r) {
          const float2 um = shfl2(v[15 - r], partner16);
          const int x = 2 * (j16 + r * M1);
#pragma unroll
          for (int h = 0; h < 2; ++h) {
            const size_t idx = row_a + (size_t)h * N + x;
            float2* th = reinterpret_cast<float2*>(d.theta + idx);
            const float2 ud = *th;
            const float2 pl = __ldg(reinterpret_cast<const float2*>(d.p_leak0 + idx));
            const float2 sk = d.s ? __ldg(reinterpret_cast<const float2*>(d.s + idx))
                                  : make_float2(1.f, 1.f);
            const float rr[2] = {h ? v[r].y : v[r].x, h ? um.y : um.x};
            const float uu[2] = {ud.x, ud.y}, pp[2] = {pl.x, pl.y}, ss[2] = {sk.x, sk.y};
            float o[2];
#pragma unroll
            for (int e = 0; e < 2; ++e) {
              const float u = fmaf((pp[e] - mu_f) * scale, rr[e], uu[e]);
              const float den = fmaf(-alpha * ss[e], u, 1.f);
              if (!(den > 0.05f)) cf_flags |= kFlagRunaway;
              o[e] = ss[e] * u / den;
              if (!isfinite(o[e])) cf_flags |= kFlagNonfinite;
            }
            *th = make_float2(o[0], o[1]);
          }
        }
      }
    }
    // the flags of the map, from every CTA
    for (int o = 16; o > 0; o >>= 1) cf_flags |= __shfl_down_sync(0xffffffffu, cf_flags, o);
    if (lane == 0) {
      red_f[warp] = 0.f;
      red_i[warp] = cf_flags;
    }
    __syncthreads();
    put_slots();
    cl_sync();
    if (rank == 0 && t == 0) {
      int ff = 0;
      for (int r = 0; r < ranks; ++r) ff |= slots->flags[r];
      vs_solve_info* inf = P.info + b;
      inf->status = (ff & kFlagRunaway) ? VS_ERR_RUNAWAY : (ff & kFlagNonfinite) ? VS_ERR_NONFINITE : VS_OK;
      inf->iterations = 0;
      inf->residual_K = 0.0;
      inf->mu_W = mu;
      inf->fell_back = 0;
    }
    // (the fixed-point path below is not compiled into this instantiation)
  } else {
  // Preconditioner and start. The source term - beta mu_p u and the
  // multiplier K / (1 - beta mu_p K) have the same fixed point for every mu_p.
  // A cold start solves the uniform mode of the die first (a scalar fixed
  // point: u = K00 (mean P_dyn + mu (1 + beta theta)), theta = u / (1 - alpha u)),
  // starts from that uniform temperature th0 instead of 0, and takes
  // mu_p = mu (1 + 2 alpha u): beta P_leak0 dtheta/du, with dtheta/du =
  // s / (1 - alpha s u)^2, averages about beta mu_p over the die, so the
  // iteration is left with the variation alone.
  float th0 = 0.f, mu_p = (float)mu;
  if ((double)beta * mu * (double)d.kmax >= 0.999) {
    status = VS_ERR_RUNAWAY;
    stop = true;
    if (cold)   // theta_0 = 0 is the result of a map stopped before its first iterate
      for (int i = t; i < kClRows * N / 4; i += kClThreads)
        *reinterpret_cast<float4*>(d.theta + (size_t)y0 * N + 4 * i) = make_float4(0.f, 0.f, 0.f, 0.f);
  } else {
    if (cold) {
      double pd_sum = 0.0;
      for (int r = 0; r < ranks; ++r) pd_sum += slots->part2[r];
      const float pdm = (float)(pd_sum / ((double)N * N)), muf = (float)mu;
      const float k00 = __ldg(d.Kt);
      if constexpr (!PHYS) {
        float ub = 0.f;
        bool ok = true;
        for (int k = 0; k < 16 && ok; ++k) {   // contracts by ~beta mu K00 per step
          const float den = fmaf(-alpha, ub, 1.f);
          ok = den > 0.05f;
          ub = k00 * fmaf(muf, fmaf(beta, __fdividef(ub, den), 1.f), pdm);
        }
        const float den = fmaf(-alpha, ub, 1.f);
        const float mp = muf * fmaf(2.f * alpha, ub, 1.f);
        if (ok && den > 0.05f && isfinite(ub) && beta * mp * d.kmax < 0.95f) {
          th0 = __fdividef(ub, den);
          mu_p = mp;
        }
      } else {
        // the same for a variant: u = K00 (mean P_dyn + mu g(theta(u))) at s = 1,
        // preconditioner b = mu g'(theta) dtheta/du there, i.e. mu_p = b / beta
        // (beta the slope the source term and the multiplier scale by)
        float ub = 0.f, tb = 0.f;
        int fl = 0;
        for (int k = 0; k < 16 && !fl; ++k) {
          tb = cl_field_theta(P, 1.f, ub, fl);
          ub = k00 * fmaf(muf, cl_leak(P, tb), pdm);
        }
        tb = cl_field_theta(P, 1.f, ub, fl);
        const float b = muf * cl_leak_slope(P, tb) * cl_field_dtheta(P, ub);
        if (!fl && isfinite(tb) && isfinite(b) && beta > 0.f && b > 0.f && b * d.kmax < 0.95f) {
          th0 = tb;
          mu_p = b / beta;
        }
      }
    }
    float r0 = 0.f;
    int f0 = 0;
    // the peers' start is already established by the barrier above
    row_phase(1, mu_p, th0, r0, f0, 0);
    cl_sync();
  }

  if (!stop) {
    {
      // spectral multiplier of this CTA's frequency pairs, with the 1 / N^2
      // of the two unnormalised inverse transforms folded in
      const float bm = beta * mu_p;
      const float inv_n2 = 1.f / ((float)N * (float)N);
#pragma unroll
      for (int i = 0; i < kKv; ++i) {
        const int it = t + i * kClThreads;
        const int q = it % N, jj = it / N;
        const float ka = kv[i].x, kb = kv[i].y;
        Ls[q * kClF + (jj ^ (q & (kClF - 1)))] =
            make_float2(__fdividef(ka, 1.f - bm * ka) * inv_n2, __fdividef(kb, 1.f - bm * kb) * inv_n2);
      }
      __syncthreads();
    }
    for (int it = 1; it <= P.max_iter; ++it) {
      col_phase();
      cl_sync();
      float resid = 0.f;
      int flags = 0;
      // from the second iterate on the decision comes before the forward
      // transform (the first rarely stops: its update is the jump from the start)
      const int early = it >= 2 ? it : 0;
      row_phase(it == 1 && cold ? 3 : 2, mu_p, th0, resid, flags, early);
      if (!early) {
        put_slots();
        cl_sync();
        decide(it);
      } else if (!stop) {
        cl_sync();
      }
      if (stop) break;
    }
  }
  if (rank == 0 && t == 0) {
    vs_solve_info* inf = P.info + b;
    inf->status = status;
    inf->iterations = iters;
    inf->residual_K = (double)prev;
    inf->mu_W = mu;
  }
  }   // fixed-point path
}


}  // namespace

bool cluster_size_ok(int n) { return n >= 32 && n <= kClMaxN; }

ClHost cluster_shape(int n) {
  switch (n) {
    case 32: return {ClShape<32>::RANKS, ClShape<32>::THREADS, ClLayout<32>::kBytes};
    case 64: return {ClShape<64>::RANKS, ClShape<64>::THREADS, ClLayout<64>::kBytes};
    case 128: return {ClShape<128>::RANKS, ClShape<128>::THREADS, ClLayout<128>::kBytes};
    default: return {ClShape<256>::RANKS, ClShape<256>::THREADS, ClLayout<256>::kBytes};
  }
}

template <int N>
ClusterFn cluster_kernel_n(int batch) {
  switch (batch) {
    case 1: return k_solve_cluster<N, 1>;
    case 4: return k_solve_cluster<N, 4>;
    default: return k_solve_cluster<N, 2>;
  }
}

ClusterFn cluster_kernel(int n, int batch) {
  switch (n) {
    case 32: return cluster_kernel_n<32>(batch);
    case 64: return cluster_kernel_n<64>(batch);
    case 128: return cluster_kernel_n<128>(batch);
    default: return cluster_kernel_n<256>(batch);
  }
}

// The physics-variant instantiation for grid side n (update-load batch 2).
ClusterFn cluster_kernel_phys(int n) {
  switch (n) {
    case 32: return k_solve_cluster<32, 2, false, true>;
    case 64: return k_solve_cluster<64, 2, false, true>;
    case 128: return k_solve_cluster<128, 2, false, true>;
    default: return k_solve_cluster<256, 2, false, true>;
  }
}

// The closed-form instantiation for grid side n (32 .. 256): one cluster per
// map over `count` maps; shared-memory attributes set once per n.
cudaError_t cluster_cf_launch(int n, const ClusterDev& P, int count, cudaStream_t s) {
  static bool attr_set[4] = {};
  ClusterFn fn = n == 32 ? k_solve_cluster<32, 2, true>
                 : n == 64 ? k_solve_cluster<64, 2, true>
                 : n == 128 ? k_solve_cluster<128, 2, true>
                            : k_solve_cluster<256, 2, true>;
  const ClHost h = cluster_shape(n);
  const int ni = __builtin_ctz((unsigned)n) - 5;
  if (!attr_set[ni]) {
    cudaError_t e = cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)h.smem);
    if (e == cudaSuccess)
      e = cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    attr_set[ni] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3((unsigned)h.ranks * (unsigned)count);
  cfg.blockDim = dim3((unsigned)h.threads);
  cfg.dynamicSmemBytes = h.smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)h.ranks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cudaLaunchKernelEx(&cfg, fn, P);
}


}  // namespace vsk
