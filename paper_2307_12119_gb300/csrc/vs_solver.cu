// Persistent batched solver of the leakage/conductivity fixed point
// (Eqs. 13-26 with the convergence loop of Sec. V-C) and of the transient
// superposition (Eqs. 27-37).
//
// One cooperative launch per solve. Every map is a set of tasks:
//   row task  : RB consecutive rows of one map
//     - inverse DCT along x of the column-phase output (transposed layout),
//     - fused update: u -> theta = s u / (1 - alpha s u), residual
//       max |theta - theta_prev|, source q = P_dyn + P_leak0
//       + beta (P_leak0 theta - mu u) (mean/variation split, Sec. IV-C),
//     - forward DCT along x, stored transposed (x-frequency major);
//   col task  : CB consecutive x-frequencies of one map
//     - forward DCT along y, multiply by the shift-invariant modified kernel
//       K / (1 - beta mu K) (Eq. 21 with alpha = 0), inverse DCT along y.
// Phases are separated by a grid barrier; after each row phase one thread
// per map decides convergence. Maps converge independently; the launch ends
// when no map is active.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <stddef.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <map>
#include <mutex>
#include <vector>

#include "vs_fft.cuh"
#include "vs_internal.cuh"
#include "vs_solve_common.cuh"
#include "vs_tc.cuh"

using namespace vsfft;
using namespace vsk;

namespace {

constexpr int kThreads = 256;
constexpr int kU = 4;          // items per thread with loads issued together
constexpr int kMaxIter = 1000;
constexpr long long kSpinLimit = 20000000LL;  // ~ seconds at ~100 ns per spin


struct MapState {
  double mu;
  float mu_f;
  float b_col, b_row;    // preconditioner coefficient of the next column / row phase
  float th0;             // uniform start of a cold map (adaptive plans)
  unsigned resid_bits;
  float prev_resid;
  int growth;
  int active;
  int status;
  int iters;
  int flags;
};

struct Ctrl {
  unsigned count;
  unsigned gen;
  unsigned abort;
  unsigned pad_;
  unsigned active[kMaxIter + 2];
};

struct PlanDev {
  const MapDesc* maps;
  const int* row_map;    // task -> map index
  const int* col_map;
  MapState* st;
  double* part;          // per row task: sum of P_leak0 (then of the iteration's data)
  double* part2;         // per row task: sum of P_dyn (adaptive plans)
  vs_solve_info* info;
  Ctrl* ctrl;
  int n_maps, row_tasks, col_tasks;
  int max_iter;
  float beta, alpha, tol;
  int stop_rule;         // VS_STOP_* (steady solves)
  int n_steps;           // transient
  int warm;              // some map has a warm start
  int window;            // transient: 0 untruncated, K >= 1 step responses settled from age K on
  int implicit;          // transient: per-step leakage fixed point
  int adaptive;          // steady FP32: a cold map starts from the die's uniform-mode
                         // temperature, preconditioned with beta mu (1 + 2 alpha u)
  float* xs;             // transient, implicit: the last source spectrum of the current step
  // physics variants (the k_solve_steady<true> instantiation); beta above is
  // then the preconditioner slope (the secant of a piecewise-linear table)
  int cond;              // VS_COND_*
  float one_me, t_amb;   // Kirchhoff: 1 - eta, T_amb
  int leak_n;            // 0: linear leakage 1 + beta theta; else table points
  float leak_x[VS_MAX_LEAK_POINTS], leak_y[VS_MAX_LEAK_POINTS];
};

// ------------------------------------------------------------ sums
// Compensated FP32 accumulation (Knuth's two-sum): hi + lo is the exact sum of
// the added values to about 1e-14 relative. FP64 adds run at a small fraction
// of the FP32 rate on this part, and the leakage sums touch every cell.
struct Sum2 {
  float hi = 0.f, lo = 0.f;
  __device__ __forceinline__ void add(float x) {
    const float t = hi + x, bp = t - hi;
    lo += (hi - (t - bp)) + (x - bp);
    hi = t;
  }
  __device__ __forceinline__ double value() const { return (double)hi + (double)lo; }
};

// ------------------------------------------------------------ physics variants
// Leakage factor g(theta): linear, or piecewise linear through the table with
// the end segments extended (Sec. II-E).
__device__ __forceinline__ float leak_factor(const PlanDev& P, float th) {
  if (P.leak_n == 0) return fmaf(P.beta, th, 1.f);
  int i = 0;
  while (i < P.leak_n - 2 && th >= P.leak_x[i + 1]) ++i;
  const float x0 = P.leak_x[i], y0 = P.leak_y[i];
  return fmaf((P.leak_y[i + 1] - y0) / (P.leak_x[i + 1] - x0), th - x0, y0);
}

// theta from the linear solution u at the field point: Eqs. 11-12, or the
// inverse Kirchhoff transform of s u for kappa ~ T^-eta (Eq. 10). Flags a base
// (1 - alpha s u, or 1 + (1 - eta) s u / T_amb) <= 0.05 as runaway.
__device__ __forceinline__ float field_theta(const PlanDev& P, float sk, float uu, int& flags) {
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

// Its inverse: the u of a temperature (warm starts).
__device__ __forceinline__ float field_u(const PlanDev& P, float sk, float t0) {
  if (P.cond == VS_COND_KIRCHHOFF)
    return P.t_amb * expm1f(P.one_me * log1pf(t0 / P.t_amb)) / (P.one_me * sk);
  return t0 / (sk * fmaf(P.alpha, t0, 1.f));
}

// ------------------------------------------------------------ grid barrier

__device__ __forceinline__ unsigned ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Returns false if the launch was aborted (a barrier timed out somewhere).
__device__ bool grid_barrier(Ctrl* c) {
  __syncthreads();
  if (threadIdx.x == 0) {
    unsigned gen = ld_acquire(&c->gen);
    __threadfence();
    unsigned arrived = atomicAdd(&c->count, 1u) + 1u;
    if (arrived == gridDim.x) {
      atomicExch(&c->count, 0u);
      __threadfence();
      atomicAdd(&c->gen, 1u);
    } else {
      long long spins = 0;
      while (ld_acquire(&c->gen) == gen) {
        if (ld_acquire(&c->abort)) break;
        __nanosleep(64);
        if (++spins > kSpinLimit) {
          atomicExch(&c->abort, 1u);
          break;
        }
      }
    }
    __threadfence();
  }
  __syncthreads();
  return ld_acquire(&c->abort) == 0u;
}

// ------------------------------------------------------------ reductions


__device__ __forceinline__ float block_max(float v, float* red) {
  for (int o = 16; o > 0; o >>= 1) v = fmaxf(v, __shfl_down_sync(0xffffffffu, v, o));
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  float r = 0.f;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r = fmaxf(r, red[i]);
  __syncthreads();
  return r;
}

__device__ __forceinline__ int block_or(int v, int* red) {
  for (int o = 16; o > 0; o >>= 1) v |= __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  int r = 0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r |= red[i];
  __syncthreads();
  return r;
}

__device__ __forceinline__ int find_map(const PlanDev& P, int task, bool row) {
  return __ldg(row ? &P.row_map[task] : &P.col_map[task]);
}

// ------------------------------------------------------------ row transforms
// Rows y0 .. y0 + rb - 1 of a map are held in buf as rb/2 interleaved pairs
// (float2 = two rows), in the digit-reversed order of the radix FFT.

// Inverse DCT along x of the rows from the transposed spectral work map.
__device__ __forceinline__ void row_inverse(const MapDesc& d, int y0, float2* buf) {
  const int n = d.n, F = d.rb >> 1, NP = padded_len(n), half = n >> 1;
  const int lgF = __ffs(F) - 1;
  const float* WT = d.work;
  const float2* tw = d.tw4n;
  const int* dr = d.digrev;
  const int total = F * (half + 1);
  for (int base = threadIdx.x; base < total; base += kU * blockDim.x) {
    float2 xk[kU], xnk[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      int it = base + u * blockDim.x;
      xk[u] = xnk[u] = make_float2(0.f, 0.f);
      if (it < total) {
        int f = it & (F - 1), k = it >> lgF;
        xk[u] = *reinterpret_cast<const float2*>(WT + (size_t)k * n + y0 + 2 * f);
        if (k != 0) xnk[u] = *reinterpret_cast<const float2*>(WT + (size_t)(n - k) * n + y0 + 2 * f);
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      int it = base + u * blockDim.x;
      if (it < total) {
        int f = it & (F - 1), k = it >> lgF, nk = n - k;
        buf[f * NP + pad(__ldg(&dr[k]))] = dct_pre(xk[u].x, xnk[u].x, xk[u].y, xnk[u].y, __ldg(&tw[k]));
        if (k != 0 && k != half)
          buf[f * NP + pad(__ldg(&dr[nk]))] = dct_pre(xnk[u].x, xk[u].x, xnk[u].y, xk[u].y, __ldg(&tw[nk]));
      }
    }
  }
  __syncthreads();
  fft_inverse(buf, n, F, NP, tw);
}

// Forward DCT along x of the rows in buf (natural Makhoul order), stored
// transposed (x-frequency major) into the spectral work map.
__device__ __forceinline__ void row_forward(const MapDesc& d, int y0, float2* buf) {
  const int n = d.n, F = d.rb >> 1, NP = padded_len(n), half = n >> 1;
  const int lgF = __ffs(F) - 1;
  float* WT = d.work;
  const float2* tw = d.tw4n;
  const int* dr = d.digrev;
  fft_forward(buf, n, F, NP, tw);
  for (int it = threadIdx.x; it < F * (half + 1); it += blockDim.x) {
    int f = it & (F - 1), k = it >> lgF, nk = n - k;
    float2 zk = buf[f * NP + pad(__ldg(&dr[k]))];
    float2 znk = buf[f * NP + pad(__ldg(&dr[k == 0 ? 0 : nk]))];
    *reinterpret_cast<float2*>(WT + (size_t)k * n + y0 + 2 * f) = dct_post(zk, znk, __ldg(&tw[k]));
    if (k != 0 && k != half)
      *reinterpret_cast<float2*>(WT + (size_t)nk * n + y0 + 2 * f) = dct_post(znk, zk, __ldg(&tw[nk]));
  }
  __syncthreads();
}

// ------------------------------------------------------------ row task
// MODE 0: steady iteration `step` (0 = initial source from theta_0 = 0,
// -1 = initial source from a warm start theta_0, -2 = mean leakage only).
// MODE 1: transient step `step` (0 = first source, n_steps = last inverse only).
// PHYS (MODE 0): the leakage factor and field-point map of the physics variants.
template <int MODE, bool PHYS = false>
__device__ void row_task(const PlanDev& P, int task, int step, float2* buf) {
  __shared__ double red_d[kThreads / 32];
  __shared__ float red_f[kThreads / 32];
  __shared__ int red_i[kThreads / 32];
  const int b = find_map(P, task, true);
  const MapDesc d = P.maps[b];
  MapState* ms = P.st + b;
  if (MODE == 0 && (step > 0 || step == -1) && !ms->active) {
    if (step == -1 && !d.theta_init) {
      // a cold map stopped before its first iterate (runaway): theta_0 = 0
      const int n = d.n, y0 = (task - d.row_off) * d.rb;
      for (int i = threadIdx.x; i < d.rb * n; i += blockDim.x) d.theta[(size_t)y0 * n + i] = 0.f;
    }
    return;
  }
  const int n = d.n, F = d.rb >> 1, NP = padded_len(n);
  const int lgn = __ffs(n) - 1;
  const int chunk = task - d.row_off;
  const int y0 = chunk * d.rb;
  const bool first = (step <= 0);
  const bool warm = (MODE == 0) && (step == -1);
  const bool muonly = (MODE == 0) && (step == -2);
  const bool last = (MODE == 1) && (step == P.n_steps);
  if (muonly) {
    // the means of the inputs: P_leak0, and P_dyn of a cold map of an adaptive plan
    const bool with_pd = P.adaptive && !d.theta_init;
    Sum2 acc, acc_d;
    const float4* l4 = reinterpret_cast<const float4*>(d.p_leak0 + (size_t)y0 * n);
    const float4* d4 = reinterpret_cast<const float4*>(d.p_dyn + (size_t)y0 * n);
#pragma unroll 4
    for (int i = threadIdx.x; i < d.rb * n / 4; i += blockDim.x) {
      const float4 a = __ldg(l4 + i);
      const float4 c = with_pd ? __ldg(d4 + i) : make_float4(0.f, 0.f, 0.f, 0.f);
      acc.add(a.x);
      acc.add(a.y);
      acc.add(a.z);
      acc.add(a.w);
      acc_d.add(c.x);
      acc_d.add(c.y);
      acc_d.add(c.z);
      acc_d.add(c.w);
    }
    double tot = block_sum(acc.value(), red_d);
    double tot_d = with_pd ? block_sum(acc_d.value(), red_d) : 0.0;
    if (threadIdx.x == 0) {
      P.part[d.part_off + chunk] = tot;
      P.part2[d.part_off + chunk] = tot_d;
    }
    __syncthreads();
    return;
  }
  // a cold map of an adaptive plan starts from the uniform temperature th0
  const bool uni = MODE == 0 && !PHYS && P.adaptive && !d.theta_init;

  if (!first) row_inverse(d, y0, buf);

  // fused elementwise update; bq is the preconditioner coefficient of the
  // source term - bq u (the next column phase multiplies by K / (1 - bq K))
  const float beta = P.beta, alpha = P.alpha;
  const float bq = (MODE == 0 && (!first || warm)) ? ms->b_row : 0.f;
  Sum2 mu_acc;           // sum of P_leak0 (first pass)
  float resid = 0.f;
  int flags = 0;
  const size_t nn = (size_t)n * n;
  const int total = F * n;
  for (int base = threadIdx.x; base < total; base += kU * blockDim.x) {
    float pl[kU][2], pd[kU][2], sk[kU][2], old[kU][2];
    float2 uv[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      int it = base + u * blockDim.x;
      uv[u] = make_float2(0.f, 0.f);
#pragma unroll
      for (int h = 0; h < 2; ++h) pl[u][h] = pd[u][h] = old[u][h] = 0.f, sk[u][h] = 1.f;
      if (it < total) {
        int f = it >> lgn, x = it & (n - 1);
        if (!first) uv[u] = buf[f * NP + pad(makhoul_pos(x, n))];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          size_t idx = (size_t)(y0 + 2 * f + h) * n + x;
          pl[u][h] = __ldg(&d.p_leak0[idx]);
          if (d.s) sk[u][h] = __ldg(&d.s[idx]);
          if (MODE == 0) {
            pd[u][h] = __ldg(&d.p_dyn[idx]);
            if (uni && (warm || step == 1)) old[u][h] = ms->th0;
            else if (!first) old[u][h] = d.theta[idx];
            else if (warm && d.theta_init) old[u][h] = __ldg(&d.theta_init[idx]);
          } else if (!last) {
            pd[u][h] = __ldg(&d.p_dyn[(size_t)step * nn + idx]);
          }
        }
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      int it = base + u * blockDim.x;
      if (it >= total) continue;
      int f = it >> lgn, x = it & (n - 1);
      float q[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        size_t idx = (size_t)(y0 + 2 * f + h) * n + x;
        float uu = h ? uv[u].y : uv[u].x;
        if (MODE == 0) {
          if (PHYS) {
            // P_dyn + P_leak0 g(theta) - beta mu u, beta the preconditioner slope
            float th = 0.f, uq = 0.f;
            if (warm) {
              th = old[u][h];
              uq = field_u(P, sk[u][h], th);
            } else if (!first) {
              th = field_theta(P, sk[u][h], uu, flags);
              uq = uu;
              if (!isfinite(th)) flags |= kFlagNonfinite;
              else resid = fmaxf(resid, fabsf(th - old[u][h]));
            } else {
              mu_acc.add(pl[u][h]);
            }
            d.theta[idx] = th;
            q[h] = fmaf(pl[u][h], leak_factor(P, th), pd[u][h]) - bq * uq;
          } else if (warm) {
            // theta_0 from the warm start (or uniform, not stored);
            // u_0 = theta_0 / (s (1 + alpha theta_0))
            float t0 = old[u][h];
            float u0 = __fdividef(t0, sk[u][h] * fmaf(alpha, t0, 1.f));
            if (!uni) d.theta[idx] = t0;
            q[h] = fmaf(beta * pl[u][h], t0, pd[u][h] + pl[u][h]) - bq * u0;
          } else if (first) {
            d.theta[idx] = 0.f;
            q[h] = pd[u][h] + pl[u][h];
            mu_acc.add(pl[u][h]);
          } else {
            float den = fmaf(-alpha * sk[u][h], uu, 1.f);
            if (!(den > 0.05f)) flags |= kFlagRunaway;
            float th = __fdividef(sk[u][h] * uu, den);   // as the cluster engine
            if (!isfinite(th)) flags |= kFlagNonfinite;
            else resid = fmaxf(resid, fabsf(th - old[u][h]));
            d.theta[idx] = th;
            q[h] = fmaf(beta * pl[u][h], th, pd[u][h] + pl[u][h]) - bq * uu;
          }
        } else {
          float th = 0.f;
          if (!first) {
            float den = fmaf(-alpha * sk[u][h], uu, 1.f);
            if (!(den > 0.05f)) flags |= kFlagRunaway;
            th = sk[u][h] * uu / den;
            if (!isfinite(th)) flags |= kFlagNonfinite;
            d.theta[(size_t)(step - 1) * nn + idx] = th;
          }
          q[h] = last ? 0.f : pd[u][h] + pl[u][h] * fmaf(beta, th, 1.f);
        }
      }
      buf[f * NP + pad(makhoul_pos(x, n))] = make_float2(q[0], q[1]);
    }
  }
  if (MODE == 0 && first && !warm) {
    double tot = block_sum(mu_acc.value(), red_d);
    if (threadIdx.x == 0) P.part[d.part_off + chunk] = tot;
  }
  if (!first || MODE == 1) {
    float r = block_max(resid, red_f);
    int fl = block_or(flags, red_i);
    if (threadIdx.x == 0) {
      if (MODE == 0 && r > 0.f) atomicMax(&ms->resid_bits, __float_as_uint(r));
      if (fl) atomicOr(&ms->flags, fl);
    }
  }
  __syncthreads();
  if (last) return;
  row_forward(d, y0, buf);
}

// ------------------------------------------------------------ column task
// MODE 1: `step` is the 1-based transient step n of the source in the work
// map. VAR: the variants (window, implicit leakage) are compiled in; then
// `commit` (implicit leakage, first iteration of a step) first folds the
// previous step's final source spectrum into the history.
template <int MODE, bool VAR = false>
__device__ void col_task(const PlanDev& P, int task, float2* buf, int step = 0, bool commit = false) {
  const int b = find_map(P, task, false);
  const MapDesc d = P.maps[b];
  MapState* ms = P.st + b;
  if (MODE == 0 && !ms->active) return;
  const int n = d.n, F = d.cb >> 1, NP = padded_len(n), half = n >> 1;
  const int lgF = __ffs(F) - 1, lgn = __ffs(n) - 1;
  const int p0 = (task - d.col_off) * d.cb;
  float* WT = d.work;
  const float2* tw = d.tw4n;
  const int* dr = d.digrev;

  const int total = F * n;
  for (int base = threadIdx.x; base < total; base += kU * blockDim.x) {
    float a[kU], c[kU];
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      int it = base + u * blockDim.x;
      a[u] = c[u] = 0.f;
      if (it < total) {
        int f = it >> lgn, j = it & (n - 1);
        a[u] = WT[(size_t)(p0 + 2 * f) * n + j];
        c[u] = WT[(size_t)(p0 + 2 * f + 1) * n + j];
      }
    }
#pragma unroll
    for (int u = 0; u < kU; ++u) {
      int it = base + u * blockDim.x;
      if (it < total) {
        int f = it >> lgn, j = it & (n - 1);
        buf[f * NP + pad(makhoul_pos(j, n))] = make_float2(a[u], c[u]);
      }
    }
  }
  __syncthreads();
  fft_forward(buf, n, F, NP, tw);

  const float inv_n2 = 1.f / ((float)n * (float)n);
  const float bm = (MODE == 0) ? ms->b_col : 0.f;
  for (int it = threadIdx.x; it < F * (half + 1); it += blockDim.x) {
    int f = it & (F - 1), k = it >> lgF, nk = n - k;
    int ia = f * NP + pad(__ldg(&dr[k]));
    int ib = f * NP + pad(__ldg(&dr[k == 0 ? 0 : nk]));
    float2 zk = buf[ia], znk = buf[ib];
    float2 xk = dct_post(zk, znk, __ldg(&tw[k]));
    float2 xnk = (k == 0) ? make_float2(0.f, 0.f) : dct_post(znk, zk, __ldg(&tw[nk]));
    const size_t ra = (size_t)(p0 + 2 * f) * n, rb = ra + n;
    float2 yk, ynk;
    if (MODE == 0) {
      float ka = __ldg(&d.Kt[ra + k]), kb = __ldg(&d.Kt[rb + k]);
      yk = make_float2(xk.x * ka / (1.f - bm * ka) * inv_n2, xk.y * kb / (1.f - bm * kb) * inv_n2);
      if (k != 0) {
        float ka2 = __ldg(&d.Kt[ra + nk]), kb2 = __ldg(&d.Kt[rb + nk]);
        ynk = make_float2(xnk.x * ka2 / (1.f - bm * ka2) * inv_n2, xnk.y * kb2 / (1.f - bm * kb2) * inv_n2);
      } else {
        ynk = make_float2(0.f, 0.f);
      }
    } else {
      // Step response of a mode: S_j = (K - A) + A (1 - rho^j) (the primary
      // alias relaxes with rho = exp(-dt / tau), the finer aliases settle in one step).
      auto mode = [&](size_t idx, float x) {
        const float A = __ldg(&d.trA[idx]), K = __ldg(&d.Kt[idx]);
        if (!VAR) {
          const float rho = __ldg(&d.trRho[idx]);
          const float w = fmaf(rho, d.state[idx] - x, x);
          d.state[idx] = w;
          return fmaf(K - A, x, A * w) * inv_n2;
        }
        if (P.window == 1) return K * x * inv_n2;               // every response settled
        const float rho = __ldg(&d.trRho[idx]);
        if (P.window == 0) {
          // untruncated: W_n = (1 - rho) X_n + rho W_{n-1};  Y = (K - A) X_n + A W_n
          float w = d.state[idx];
          if (P.implicit) {
            if (commit) {
              w = fmaf(rho, w - P.xs[idx], P.xs[idx]);
              d.state[idx] = w;
            }
            P.xs[idx] = x;
            return fmaf(K - A, x, A * fmaf(rho, w - x, x)) * inv_n2;
          }
          w = fmaf(rho, w - x, x);
          d.state[idx] = w;
          return fmaf(K - A, x, A * w) * inv_n2;
        }
        // window K: S_j = K for j >= K, so
        //   Y_n = K X_n - A sum_{j=1}^{K-1} rho^j (X_{n-j+1} - X_{n-j})
        // from a ring of the last K - 1 sources (X_m in slot m mod (K - 1)).
        const int R = P.window - 1;
        const size_t nn = (size_t)d.n * d.n;
        auto slot = [&](int m) { return (size_t)(((m % R) + R) % R) * nn + idx; };
        if (P.implicit && commit) d.state[slot(step - 1)] = P.xs[idx];
        float acc = 0.f, r = rho, prev = x;
        for (int j = 1; j <= R; ++j) {
          const float older = d.state[slot(step - j)];
          acc = fmaf(r, prev - older, acc);
          prev = older;
          r *= rho;
        }
        if (P.implicit) P.xs[idx] = x;
        else d.state[slot(step)] = x;
        return fmaf(K, x, -A * acc) * inv_n2;
      };
      yk = make_float2(mode(ra + k, xk.x), mode(rb + k, xk.y));
      if (k != 0 && k != half) ynk = make_float2(mode(ra + nk, xnk.x), mode(rb + nk, xnk.y));
      else if (k == half) ynk = yk;
      else ynk = make_float2(0.f, 0.f);
    }
    if (MODE == 0 && k == half) ynk = yk;
    buf[ia] = dct_pre(yk.x, ynk.x, yk.y, ynk.y, __ldg(&tw[k]));
    if (k != 0 && k != half) buf[ib] = dct_pre(ynk.x, yk.x, ynk.y, yk.y, __ldg(&tw[nk]));
  }
  __syncthreads();
  fft_inverse(buf, n, F, NP, tw);
  for (int it = threadIdx.x; it < F * n; it += blockDim.x) {
    int f = it >> lgn, j = it & (n - 1);
    float2 v = buf[f * NP + pad(makhoul_pos(j, n))];
    WT[(size_t)(p0 + 2 * f) * n + j] = v.x;
    WT[(size_t)(p0 + 2 * f + 1) * n + j] = v.y;
  }
  __syncthreads();
}

// ------------------------------------------------------------ decision phase
__device__ void write_info(const PlanDev& P, int b, const MapState& s) {
  vs_solve_info* inf = P.info + b;
  inf->status = s.status;
  inf->iterations = s.iters;
  inf->residual_K = (double)s.prev_resid;
  inf->mu_W = s.mu;
}

__device__ void decide(const PlanDev& P, int it) {
  for (int b = blockIdx.x * blockDim.x + threadIdx.x; b < P.n_maps; b += gridDim.x * blockDim.x) {
    MapState s = P.st[b];
    const MapDesc& d = P.maps[b];
    if (it == 0) {
      int tasks = d.n / d.rb;
      double sum = 0.0;
      for (int i = 0; i < tasks; ++i) sum += P.part[d.part_off + i];
      s.mu = sum / ((double)d.n * d.n);
      s.mu_f = (float)s.mu;
      s.b_col = s.b_row = P.beta * s.mu_f;
      s.th0 = 0.f;
      s.active = 1;
      s.status = VS_OK;
      s.iters = 0;
      s.prev_resid = INFINITY;
      if ((double)P.beta * s.mu * (double)d.kmax >= 0.999) {
        s.active = 0;
        s.status = VS_ERR_RUNAWAY;
      } else if (P.adaptive && !d.theta_init) {
        // Uniform mode of the die (a scalar fixed point: u = K00 (mean P_dyn +
        // mu (1 + beta theta)), theta = u / (1 - alpha u)): the cold map starts
        // from that uniform theta and preconditions with beta mu (1 + 2 alpha u),
        // about the mean of beta P_leak0 dtheta/du (dtheta/du = s / (1 - alpha s u)^2).
        double sd = 0.0;
        for (int i = 0; i < tasks; ++i) sd += P.part2[d.part_off + i];
        const float pdm = (float)(sd / ((double)d.n * d.n)), muf = s.mu_f;
        const float k00 = __ldg(d.Kt), alpha = P.alpha, beta = P.beta;
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
          s.th0 = __fdividef(ub, den);
          s.b_col = s.b_row = beta * mp;
        }
      }
    } else {
      if (!s.active) continue;
      float r = __uint_as_float(s.resid_bits);
      s.iters = it;
      if (s.flags & kFlagNonfinite) {
        s.active = 0;
        s.status = VS_ERR_NONFINITE;
      } else if (s.flags & kFlagRunaway) {
        s.active = 0;
        s.status = VS_ERR_RUNAWAY;
      } else if (converged(r, s.prev_resid, it, P.tol, P.stop_rule)) {
        s.active = 0;
        s.status = VS_OK;
      } else {
        s.growth = (it > 2 && r > s.prev_resid) ? s.growth + 1 : 0;
        if (it >= P.max_iter || s.growth >= 5) {
          s.active = 0;
          s.status = VS_ERR_NO_CONVERGENCE;
        }
      }
      s.prev_resid = r;
    }
    s.resid_bits = 0u;
    P.st[b] = s;
    write_info(P, b, s);
    if (s.active) atomicAdd(&P.ctrl->active[it], 1u);
  }
}

template <bool PHYS>
__global__ void __launch_bounds__(kThreads, 3) k_solve_steady(PlanDev P) {
  extern __shared__ float2 smem[];
  // two passes before the iterations (the means, then the first source from
  // theta_0) for warm starts and for the uniform start of adaptive plans
  const bool two = P.warm || (P.adaptive && !PHYS);
  for (int t = blockIdx.x; t < P.row_tasks; t += gridDim.x) row_task<0, PHYS>(P, t, two ? -2 : 0, smem);
  if (!grid_barrier(P.ctrl)) return;
  decide(P, 0);
  if (!grid_barrier(P.ctrl)) return;
  if (two) {
    for (int t = blockIdx.x; t < P.row_tasks; t += gridDim.x) row_task<0, PHYS>(P, t, -1, smem);
    if (!grid_barrier(P.ctrl)) return;
  }
  if (ld_acquire(&P.ctrl->active[0]) == 0u) return;
  for (int it = 1; it <= P.max_iter; ++it) {
    for (int t = blockIdx.x; t < P.col_tasks; t += gridDim.x) col_task<0>(P, t, smem);
    if (!grid_barrier(P.ctrl)) return;
    for (int t = blockIdx.x; t < P.row_tasks; t += gridDim.x) row_task<0, PHYS>(P, t, it, smem);
    if (!grid_barrier(P.ctrl)) return;
    decide(P, it);
    if (!grid_barrier(P.ctrl)) return;
    if (ld_acquire(&P.ctrl->active[it]) == 0u) break;
  }
}

// ------------------------------------------------------------ transient, implicit leakage
// Step s (0-based), iteration `it`: theta = phi(u) of the column phase's output
// into theta[s]; max |theta - previous iterate| into *slot (the first
// iterate of step s starts from theta_{s-1}, or 0).
__device__ __noinline__ void row_tr_update(const PlanDev& P, int task, int s, int it, unsigned* slot,
                              float2* buf) {
  __shared__ float red_f[kThreads / 32];
  __shared__ int red_i[kThreads / 32];
  const int b = find_map(P, task, true);
  const MapDesc d = P.maps[b];
  const int n = d.n, F = d.rb >> 1, NP = padded_len(n), lgn = __ffs(n) - 1;
  const int y0 = (task - d.row_off) * d.rb;
  const size_t nn = (size_t)n * n;
  row_inverse(d, y0, buf);
  float* th_cur = d.theta + (size_t)s * nn;
  const float* th_prev = (it > 1) ? th_cur : (s > 0 ? th_cur - nn : nullptr);
  const float alpha = P.alpha;
  float resid = 0.f;
  int flags = 0;
  for (int i = threadIdx.x; i < F * n; i += blockDim.x) {
    const int f = i >> lgn, x = i & (n - 1);
    const float2 uv = buf[f * NP + pad(makhoul_pos(x, n))];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const size_t idx = (size_t)(y0 + 2 * f + h) * n + x;
      const float uu = h ? uv.y : uv.x;
      const float sk = d.s ? __ldg(&d.s[idx]) : 1.f;
      const float den = fmaf(-alpha * sk, uu, 1.f);
      if (!(den > 0.05f)) flags |= kFlagRunaway;
      const float th = sk * uu / den;
      const float old = th_prev ? th_prev[idx] : 0.f;
      if (!isfinite(th)) flags |= kFlagNonfinite;
      else resid = fmaxf(resid, fabsf(th - old));
      th_cur[idx] = th;
    }
  }
  const float r = block_max(resid, red_f);
  const int fl = block_or(flags, red_i);
  if (threadIdx.x == 0) {
    if (r > 0.f) atomicMax(slot, __float_as_uint(r));
    if (fl) atomicOr(&P.st[b].flags, fl);
  }
  __syncthreads();
}

// Source q = P_dyn[src] + P_leak0 (1 + beta theta[s]) (theta = 0 for s < 0),
// forward DCT along x into the work map.
__device__ __noinline__ void row_tr_source(const PlanDev& P, int task, int src, int s, float2* buf) {
  const int b = find_map(P, task, true);
  const MapDesc d = P.maps[b];
  const int n = d.n, F = d.rb >> 1, NP = padded_len(n), lgn = __ffs(n) - 1;
  const int y0 = (task - d.row_off) * d.rb;
  const size_t nn = (size_t)n * n;
  const float* th = s >= 0 ? d.theta + (size_t)s * nn : nullptr;
  const float* pd = d.p_dyn + (size_t)src * nn;
  for (int i = threadIdx.x; i < F * n; i += blockDim.x) {
    const int f = i >> lgn, x = i & (n - 1);
    float q[2];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const size_t idx = (size_t)(y0 + 2 * f + h) * n + x;
      const float t = th ? th[idx] : 0.f;
      q[h] = __ldg(&pd[idx]) + __ldg(&d.p_leak0[idx]) * fmaf(P.beta, t, 1.f);
    }
    buf[f * NP + pad(makhoul_pos(x, n))] = make_float2(q[0], q[1]);
  }
  __syncthreads();
  row_forward(d, y0, buf);
}

// Lagged leakage: P_n = P_dyn,n + P_leak0 (1 + beta theta_{n-1}), one column
// and one row phase per step.
template <bool VAR>
__device__ __forceinline__ bool transient_lagged(const PlanDev& P, float2* smem) {
  for (int t = blockIdx.x; t < P.row_tasks; t += gridDim.x) row_task<1>(P, t, 0, smem);
  if (!grid_barrier(P.ctrl)) return false;
  for (int step = 1; step <= P.n_steps; ++step) {
    for (int t = blockIdx.x; t < P.col_tasks; t += gridDim.x) col_task<1, VAR>(P, t, smem, step);
    if (!grid_barrier(P.ctrl)) return false;
    for (int t = blockIdx.x; t < P.row_tasks; t += gridDim.x) row_task<1>(P, t, step, smem);
    if (!grid_barrier(P.ctrl)) return false;
  }
  return true;
}

// Implicit leakage: P_n = P_dyn,n + P_leak0 (1 + beta theta_n); every step
// iterates theta <- phi(u_n(P_n(theta))) from theta_{n-1} until the stopping
// rule holds (the change <= tol, or its error estimate from the step's last
// two changes) or max_iter iterations. The history takes the source of the
// last iteration. Every block reads the same residual word after the
// barrier, so all take the same decision. The plan holds one map.
__device__ __noinline__ bool transient_implicit(const PlanDev& P, float2* smem) {
  unsigned* slot = P.ctrl->active;          // two residual words, used alternately
  MapState* ms = P.st;
  for (int t = blockIdx.x; t < P.row_tasks; t += gridDim.x) row_tr_source(P, t, 0, -1, smem);
  if (!grid_barrier(P.ctrl)) return false;
  int g = 0;
  for (int s = 0; s < P.n_steps; ++s) {
    float prev_r = INFINITY;   // the step's previous change (the same in every block)
    for (int it = 1; it <= P.max_iter; ++it) {
      const int cur = g & 1;
      ++g;
      for (int t = blockIdx.x; t < P.col_tasks; t += gridDim.x)
        col_task<1, true>(P, t, smem, s + 1, it == 1 && s > 0);
      if (!grid_barrier(P.ctrl)) return false;
      for (int t = blockIdx.x; t < P.row_tasks; t += gridDim.x)
        row_tr_update(P, t, s, it, slot + cur, smem);
      if (!grid_barrier(P.ctrl)) return false;
      const float r = __uint_as_float(ld_acquire(slot + cur));
      const bool bad = ld_acquire(reinterpret_cast<const unsigned*>(&ms->flags)) & kFlagNonfinite;
      const bool conv = converged(r, prev_r, it, P.tol, P.stop_rule);
      const bool done = conv || it == P.max_iter || bad;
      prev_r = r;
      if (blockIdx.x == 0 && threadIdx.x == 0) {
        // every block read the other word one iteration ago, before this
        // iteration's barriers
        slot[cur ^ 1] = 0u;
        if (done) {
          ms->iters += it;
          ms->prev_resid = fmaxf(ms->prev_resid, r);
          if (!conv) ms->growth = 1;         // a step ended unconverged
        }
      }
      if (done && s == P.n_steps - 1) break;
      for (int t = blockIdx.x; t < P.row_tasks; t += gridDim.x)
        row_tr_source(P, t, done ? s + 1 : s, s, smem);
      if (!grid_barrier(P.ctrl)) return false;
      if (done) break;
    }
  }
  return true;
}

__device__ __forceinline__ void transient_info(const PlanDev& P) {
  if (blockIdx.x == 0 && threadIdx.x == 0) {
    for (int b = 0; b < P.n_maps; ++b) {
      MapState s = P.st[b];
      s.status = (s.flags & kFlagNonfinite) ? VS_ERR_NONFINITE
                 : (s.flags & kFlagRunaway) ? VS_ERR_RUNAWAY
                 : (P.implicit && s.growth) ? VS_ERR_NO_CONVERGENCE : VS_OK;
      if (!P.implicit) {
        s.iters = P.n_steps;
        s.prev_resid = 0.f;
      }
      s.mu = 0.0;
      P.st[b] = s;
      write_info(P, b, s);
    }
  }
}

// Untruncated superposition with lagged leakage.
__global__ void __launch_bounds__(kThreads, 3) k_solve_transient(PlanDev P) {
  extern __shared__ float2 smem[];
  if (transient_lagged<false>(P, smem)) transient_info(P);
}

// The variants: a window of settled responses and/or implicit leakage.
__global__ void __launch_bounds__(kThreads, 3) k_solve_transient_var(PlanDev P) {
  extern __shared__ float2 smem[];
  if (P.implicit ? transient_implicit(P, smem) : transient_lagged<true>(P, smem)) transient_info(P);
}

__global__ void k_twiddles(int n, float2* tw) {
  int e = blockIdx.x * blockDim.x + threadIdx.x;
  if (e >= 4 * n) return;
  double sn, cs;
  sincospi(-(double)e / (2.0 * n), &sn, &cs);
  tw[e] = make_float2((float)cs, (float)sn);
}

// ------------------------------------------------------------ tensor-core path
// Split-precision cosine transforms on tcgen05 (BF16 hi/lo, FP32 accumulate).
// One 1-D transform of 128 rows of a map is a GEMM D[128][n] = A[128][n] B^T:
// A = map data (split x = hi + lo on the fly), B = the DCT matrix (hi/lo
// pre-split, pre-tiled in core-matrix order). The output columns are produced
// in chunks of N = min(n, 256) (one TMEM accumulator of 128 lanes x N FP32
// columns), each with the full K = n loop. Three MMAs per
// K-step: A_hi B_hi + A_hi B_lo + A_lo B_hi (the lo*lo term, ~2^-16 relative,
// is dropped). Per iteration four passes (rows fwd, columns fwd, columns inv,
// rows inv) with the spectral multiply and the leakage/conductivity update in
// the epilogues; the fixed-point control is the same as the SIMT path.

constexpr int kTcChunkK = 64;
// A tcgen05 kernel is held to one CTA per SM (its CTA owns the SM's tensor
// memory), so latency is hidden inside the CTA: 16 warps.
constexpr int kTcThreads = 512;
constexpr int kTcABytes = 128 * kTcChunkK * 2;   // one of A hi / lo
constexpr int kTcStageBytes = 2 * kTcABytes + 2 * 256 * kTcChunkK * 2;  // A hi/lo + B hi/lo (N <= 256)
constexpr long long kTcWaitLimit = 20000000LL;

struct TcSmem {
  uint8_t stage[2][kTcStageBytes];
  uint64_t full[2];
  uint64_t done[2];
  uint64_t fin;
  uint32_t tmem_base;
  uint32_t err;
};

struct TcCtx {
  TcSmem* sm;
  uint32_t tmem;
  int uses[2];
  int chunk;
  int fin_uses;
};

enum TcPass { kTcRowFwdFirst = 0, kTcRowFwd = 1, kTcColFwd = 2, kTcColInv = 3, kTcRowInv = 4,
              kTcMu = 5, kTcWarm = 6 };

// Producer: A chunk [128 rows][64 k], A[m][k] = G[(row0 + m) * ld + k0 + k]
// (+ G2 for the first source P_dyn + P_leak0), split into BF16 hi/lo and
// written in core-matrix order. A warp covers 16 rows x 8 k of one core
// column: 8-byte stores, two wavefronts, no bank conflicts. All loads of a
// thread are issued before the conversions.
constexpr int kTcPer = 128 * kTcChunkK / 4 / kTcThreads;   // float4 items per thread per chunk

// item u of this thread -> (k core kk, row m, half h); a warp covers 16 rows of
// one k core, so the 8-byte stores below fill whole wavefronts.
__device__ __forceinline__ void tc_item(int u, int& kk, int& m, int& h) {
  int i = threadIdx.x + u * kTcThreads;
  kk = i >> 8;
  int rem = i & 255;
  m = rem >> 1;
  h = rem & 1;
}

// Loads of one A chunk into registers (A[m][k] = G[(row0 + m) * ld + k0 + k],
// plus G2 for the first source P_dyn + P_leak0).
__device__ __forceinline__ void tc_load(float4* v, const float* G, int ld, int row0, int k0,
                                        const float* G2) {
#pragma unroll
  for (int u = 0; u < kTcPer; ++u) {
    int kk, m, h;
    tc_item(u, kk, m, h);
    size_t g = (size_t)(row0 + m) * ld + k0 + kk * 8 + h * 4;
    v[u] = *reinterpret_cast<const float4*>(G + g);
    if (G2) {
      float4 w = __ldg(reinterpret_cast<const float4*>(G2 + g));
      v[u].x += w.x; v[u].y += w.y; v[u].z += w.z; v[u].w += w.w;
    }
  }
}

// Split into BF16 hi/lo and store in core-matrix order.
__device__ __forceinline__ void tc_store(uint8_t* st, const float4* v) {
  uint8_t* hi = st;
  uint8_t* lo = st + kTcABytes;
#pragma unroll
  for (int u = 0; u < kTcPer; ++u) {
    int kk, m, h;
    tc_item(u, kk, m, h);
    __nv_bfloat16 h0, h1, h2, h3, l0, l1, l2, l3;
    vstc::split_bf16(v[u].x, h0, l0);
    vstc::split_bf16(v[u].y, h1, l1);
    vstc::split_bf16(v[u].z, h2, l2);
    vstc::split_bf16(v[u].w, h3, l3);
    uint32_t off = vstc::core_off(m, kk * 8 + h * 4, kTcChunkK);
    __nv_bfloat162 a = __halves2bfloat162(h0, h1), b = __halves2bfloat162(h2, h3);
    __nv_bfloat162 c = __halves2bfloat162(l0, l1), d = __halves2bfloat162(l2, l3);
    *reinterpret_cast<uint2*>(hi + off) =
        make_uint2(*reinterpret_cast<uint32_t*>(&a), *reinterpret_cast<uint32_t*>(&b));
    *reinterpret_cast<uint2*>(lo + off) =
        make_uint2(*reinterpret_cast<uint32_t*>(&c), *reinterpret_cast<uint32_t*>(&d));
  }
}

// One 128-row GEMM over K = `K` into TMEM columns [0, N) (N <= 256); Bg is the
// pre-tiled B of this output chunk. Returns false on a wait timeout.
__device__ bool tc_gemm(TcCtx& c, int K, int N, const uint8_t* Bg, const float* G, int ld,
                        int row0, const float* G2) {
  const int nk = K / kTcChunkK;
  const uint32_t idesc = vstc::idesc_bf16(128, N);
  const uint32_t bbytes = (uint32_t)N * kTcChunkK * 2;     // one of hi / lo
  float4 vnext[kTcPer];
  tc_load(vnext, G, ld, row0, 0, G2);
  for (int kc = 0; kc < nk; ++kc) {
    const int s = c.chunk & 1;
    float4 v[kTcPer];
#pragma unroll
    for (int u = 0; u < kTcPer; ++u) v[u] = vnext[u];
    if (kc + 1 < nk) tc_load(vnext, G, ld, row0, (kc + 1) * kTcChunkK, G2);   // in flight
    if (c.uses[s] > 0 && !vstc::mbar_wait(&c.sm->done[s], (c.uses[s] - 1) & 1, kTcWaitLimit))
      return false;
    uint8_t* st = c.sm->stage[s];
    uint8_t* bst = st + 2 * kTcABytes;
    if (threadIdx.x == 0) {
      vstc::mbar_arrive_expect_tx(&c.sm->full[s], 2 * bbytes);
      const uint8_t* src = Bg + (size_t)kc * 2 * bbytes;
      vstc::bulk_g2s(bst, src, bbytes, &c.sm->full[s]);                       // B hi
      vstc::bulk_g2s(bst + bbytes, src + bbytes, bbytes, &c.sm->full[s]);     // B lo
    }
    tc_store(st, v);
    vstc::fence_proxy_async_smem();
    __syncthreads();
    if (threadIdx.x == 0) {
      bool landed = vstc::mbar_wait(&c.sm->full[s], c.uses[s] & 1, kTcWaitLimit);
      vstc::tc_fence_after();
      if (landed) {
        const uint32_t a0 = vstc::smem_u32(st), b0 = vstc::smem_u32(bst);
        const uint32_t sbo = (kTcChunkK / 8) * 128;
#pragma unroll
        for (int ks = 0; ks < kTcChunkK / 16; ++ks) {
          const uint32_t o = ks * 256;
          uint64_t ah = vstc::smem_desc(a0 + o, 128, sbo);
          uint64_t al = vstc::smem_desc(a0 + kTcABytes + o, 128, sbo);
          uint64_t bh = vstc::smem_desc(b0 + o, 128, sbo);
          uint64_t bl = vstc::smem_desc(b0 + bbytes + o, 128, sbo);
          vstc::mma_bf16(c.tmem, ah, bh, idesc, (kc > 0 || ks > 0) ? 1u : 0u);
          vstc::mma_bf16(c.tmem, ah, bl, idesc, 1u);
          vstc::mma_bf16(c.tmem, al, bh, idesc, 1u);
        }
      } else {
        c.sm->err = 1u;
      }
      vstc::mma_commit(&c.sm->done[s]);
    }
    c.uses[s]++;
    c.chunk++;
  }
  const int sl = (c.chunk - 1) & 1;
  bool ok = vstc::mbar_wait(&c.sm->done[sl], (c.uses[sl] - 1) & 1, kTcWaitLimit);
  vstc::tc_fence_after();
  __syncthreads();
  return ok && c.sm->err == 0u;
}

// Epilogue traversal: warp w reads TMEM lanes 32 (w % 4) .. + 31 (tile rows)
// and column quarter (w / 4) of the N columns, 32 columns at a time.
template <class Op>
__device__ __forceinline__ void tc_epilogue(const TcCtx& c, int N, Op op) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int m = 32 * (w & 3) + lane;
  const int quarter = N >> 2;
  const int g = w >> 2;
  for (int c0 = g * quarter; c0 < (g + 1) * quarter; c0 += 32) {
    float v[32];
    vstc::tmem_ld32(c.tmem + ((uint32_t)(32 * (w & 3)) << 16) + (uint32_t)c0, v);
    op(m, c0, v);
  }
}

// Row-wise epilogue: each warp moves its 32 x 32 TMEM block through shared
// memory (`scratch`, 16 warps x 32 x 33 floats) and then walks it one tile
// row at a time with lane = column, so global loads and stores of the fused
// update are coalesced and independent across rows.
template <class Op>
__device__ __forceinline__ void tc_epilogue_rows(const TcCtx& c, int N, float* scratch, Op op) {
  const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const int q = w & 3;
  const int quarter = N >> 2;
  const int g = w >> 2;
  float* tile = scratch + w * (32 * 33);
  for (int c0 = g * quarter; c0 < (g + 1) * quarter; c0 += 32) {
    float v[32];
    vstc::tmem_ld32(c.tmem + ((uint32_t)(32 * q) << 16) + (uint32_t)c0, v);
#pragma unroll
    for (int j = 0; j < 32; ++j) tile[lane * 33 + j] = v[j];
    __syncwarp();
#pragma unroll 8
    for (int r = 0; r < 32; ++r) op(32 * q + r, c0 + lane, tile[r * 33 + lane]);
    __syncwarp();
  }
}

// Transposed store of a thread's 32 columns: out[(c0 + i) * ld + row]; the
// 32 lanes of a warp hold consecutive rows, so each store is one 128-B line.
__device__ __forceinline__ void store32_t(float* out, int ld, int c0, int row, const float* v) {
#pragma unroll
  for (int i = 0; i < 32; ++i) out[(size_t)(c0 + i) * ld + row] = v[i];
}

__device__ __forceinline__ void store32(float* dst, const float* v) {
#pragma unroll
  for (int i = 0; i < 32; i += 4)
    *reinterpret_cast<float4*>(dst + i) = make_float4(v[i], v[i + 1], v[i + 2], v[i + 3]);
}

// One task of a pass: rows [row0, row0+128) of map b.
__device__ bool tc_task(const PlanDev& P, TcCtx& c, int pass, int task) {
  __shared__ double red_d[kTcThreads / 32];
  __shared__ float red_f[kTcThreads / 32];
  __shared__ int red_i[kTcThreads / 32];
  const int b = __ldg(&P.row_map[task]);
  const MapDesc d = P.maps[b];
  MapState* ms = P.st + b;
  const bool first = pass == kTcRowFwdFirst;
  if (!first && pass != kTcMu && !ms->active) return true;
  const int n = d.n;
  const int tile = task - d.row_off;
  const int r0 = tile * 128;
  bool ok = true;
  Sum2 mu_acc;
  float resid = 0.f;
  int flags = 0;
  if (pass == kTcMu || pass == kTcWarm) {
    // warm start: mean leakage of the tile, then the first source from theta_0
    const float beta = P.beta, alpha = P.alpha, mu = ms->mu_f;
    for (int i = threadIdx.x; i < 128 * n; i += blockDim.x) {
      size_t idx = (size_t)r0 * n + i;
      float pl = __ldg(&d.p_leak0[idx]);
      if (pass == kTcMu) {
        mu_acc.add(pl);
      } else {
        float t0 = d.theta_init ? __ldg(&d.theta_init[idx]) : 0.f;
        float sk = d.s ? __ldg(&d.s[idx]) : 1.f;
        float u0 = t0 / (sk * fmaf(alpha, t0, 1.f));
        d.theta[idx] = t0;
        d.work2[idx] = __ldg(&d.p_dyn[idx]) + pl + beta * fmaf(pl, t0, -mu * u0);
      }
    }
    if (pass == kTcMu) {
      double tot = block_sum(mu_acc.value(), red_d);
      if (threadIdx.x == 0) P.part[d.part_off + tile] = tot;
    }
    __syncthreads();
    return true;
  }
  // output chunks of NB columns; B of chunk nc starts nc * bstride bytes in
  const int NB = n < 256 ? n : 256;
  const size_t bstride = (size_t)(n / kTcChunkK) * 2 * NB * kTcChunkK * 2;
  float* scratch = reinterpret_cast<float*>(c.sm->stage[0]);
  for (int nc = 0; nc < n / NB && ok; ++nc) {
    const int n0 = nc * NB;
    if (nc > 0) {
      // TMEM and the stage-0 epilogue scratch are reused by the next chunk
      vstc::fence_proxy_async_smem();
      vstc::tc_fence_before();
      __syncthreads();
    }
    if (pass == kTcRowFwdFirst || pass == kTcRowFwd) {
      // rows forward: A[y][x] = q (first: P_dyn + P_leak0), B = C -> R[y][p], stored as RT[p][y]
      if (first) ok = tc_gemm(c, n, NB, d.tcf + nc * bstride, d.p_dyn, n, r0, d.p_leak0);
      else ok = tc_gemm(c, n, NB, d.tcf + nc * bstride, d.work2, n, r0, nullptr);
      tc_epilogue(c, NB, [&](int m, int c0, float* v) { store32_t(d.work, n, n0 + c0, r0 + m, v); });
    } else if (pass == kTcColFwd) {
      // columns forward: A[p][y] = RT, B = C -> X[p][q]; x K/(1-beta mu K) -> Y[p][q]
      ok = tc_gemm(c, n, NB, d.tcf + nc * bstride, d.work, n, r0, nullptr);
      const float bm = P.beta * ms->mu_f;
      tc_epilogue_rows(c, NB, scratch, [&](int m, int col, float val) {
        size_t idx = (size_t)(r0 + m) * n + n0 + col;
        float k = __ldg(&d.Kt[idx]);
        d.work2[idx] = val * k / (1.f - bm * k);
      });
    } else if (pass == kTcColInv) {
      // columns inverse: A[p][q] = Y, B = Ci -> ZT[p][y], stored as Z[y][p]
      ok = tc_gemm(c, n, NB, d.tci + nc * bstride, d.work2, n, r0, nullptr);
      tc_epilogue(c, NB, [&](int m, int c0, float* v) { store32_t(d.work, n, n0 + c0, r0 + m, v); });
    } else {
      // rows inverse: A[y][p] = Z, B = Ci -> u[y][x]; fused update -> q[y][x]
      ok = tc_gemm(c, n, NB, d.tci + nc * bstride, d.work, n, r0, nullptr);
      const float beta = P.beta, alpha = P.alpha, mu = ms->mu_f;
      tc_epilogue_rows(c, NB, scratch, [&](int m, int col, float u) {
        size_t idx = (size_t)(r0 + m) * n + n0 + col;
        float pd = __ldg(&d.p_dyn[idx]);
        float pl = __ldg(&d.p_leak0[idx]);
        float sk = d.s ? __ldg(&d.s[idx]) : 1.f;
        float old = d.theta[idx];
        float den = fmaf(-alpha * sk, u, 1.f);
        if (!(den > 0.05f)) flags |= kFlagRunaway;
        float th = sk * u / den;
        if (!isfinite(th)) flags |= kFlagNonfinite;
        else resid = fmaxf(resid, fabsf(th - old));
        d.theta[idx] = th;
        d.work2[idx] = pd + pl + beta * fmaf(pl, th, -mu * u);
      });
    }
  }
  if (first) {
    // theta_0 = 0 and the partial sum of P_leak0 over the tile (coalesced)
    for (int i = threadIdx.x; i < 128 * n / 4; i += blockDim.x) {
      size_t idx = (size_t)r0 * n + 4 * (size_t)i;
      *reinterpret_cast<float4*>(d.theta + idx) = make_float4(0.f, 0.f, 0.f, 0.f);
      float4 w4 = __ldg(reinterpret_cast<const float4*>(d.p_leak0 + idx));
      mu_acc.add(w4.x);
      mu_acc.add(w4.y);
      mu_acc.add(w4.z);
      mu_acc.add(w4.w);
    }
  }
  // the epilogue scratch (stage 0) is refilled by the async proxy next
  vstc::fence_proxy_async_smem();
  vstc::tc_fence_before();
  if (first) {
    double tot = block_sum(mu_acc.value(), red_d);
    if (threadIdx.x == 0) P.part[d.part_off + tile] = tot;
  } else if (pass == kTcRowInv) {
    float r = block_max(resid, red_f);
    int fl = block_or(flags, red_i);
    if (threadIdx.x == 0) {
      if (r > 0.f) atomicMax(&ms->resid_bits, __float_as_uint(r));
      if (fl) atomicOr(&ms->flags, fl);
    }
  }
  __syncthreads();
  return ok;
}

__device__ void tc_finish(TcCtx& c) {
  // wait (bounded) for every tcgen05 op issued by thread 0, then free TMEM
  if (threadIdx.x == 0) {
    vstc::mma_commit(&c.sm->fin);
    vstc::mbar_wait(&c.sm->fin, c.fin_uses & 1, kTcWaitLimit);
  }
  c.fin_uses++;
  vstc::tc_fence_before();
  __syncthreads();
  vstc::tc_fence_after();
  if ((threadIdx.x >> 5) == 0) vstc::tmem_dealloc(c.tmem, 256);
}

__global__ void __launch_bounds__(kTcThreads, 1) k_solve_steady_tc(PlanDev P) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  TcSmem* sm = reinterpret_cast<TcSmem*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  if (threadIdx.x == 0) {
    vstc::mbar_init(&sm->full[0], 1);
    vstc::mbar_init(&sm->full[1], 1);
    vstc::mbar_init(&sm->done[0], 1);
    vstc::mbar_init(&sm->done[1], 1);
    vstc::mbar_init(&sm->fin, 1);
    vstc::mbar_fence_init();
    sm->err = 0u;
  }
  if ((threadIdx.x >> 5) == 0) vstc::tmem_alloc(&sm->tmem_base, 256);
  vstc::tc_fence_before();
  __syncthreads();
  vstc::tc_fence_after();
  TcCtx c;
  c.sm = sm;
  c.tmem = sm->tmem_base;
  c.uses[0] = c.uses[1] = 0;
  c.chunk = 0;
  c.fin_uses = 0;
  bool alive = true;
  auto pass_all = [&](int pass) {
    for (int t = blockIdx.x; t < P.row_tasks && alive; t += gridDim.x)
      if (!tc_task(P, c, pass, t)) {
        atomicExch(&P.ctrl->abort, 1u);
        alive = false;
      }
  };
  pass_all(P.warm ? kTcMu : kTcRowFwdFirst);
  if (alive) alive = grid_barrier(P.ctrl);
  if (alive) decide(P, 0);
  if (alive) alive = grid_barrier(P.ctrl);
  if (alive && P.warm && ld_acquire(&P.ctrl->active[0]) != 0u) {
    pass_all(kTcWarm);
    if (alive) alive = grid_barrier(P.ctrl);
    if (alive) pass_all(kTcRowFwd);
    if (alive) alive = grid_barrier(P.ctrl);
  }
  if (alive && ld_acquire(&P.ctrl->active[0]) != 0u) {
    for (int it = 1; it <= P.max_iter && alive; ++it) {
      pass_all(kTcColFwd);
      if (alive) alive = grid_barrier(P.ctrl);
      if (alive) pass_all(kTcColInv);
      if (alive) alive = grid_barrier(P.ctrl);
      if (alive) pass_all(kTcRowInv);
      if (alive) alive = grid_barrier(P.ctrl);
      if (alive) decide(P, it);
      if (alive) alive = grid_barrier(P.ctrl);
      if (!alive || ld_acquire(&P.ctrl->active[it]) == 0u) break;
      pass_all(kTcRowFwd);
      if (alive) alive = grid_barrier(P.ctrl);
    }
  }
  tc_finish(c);
}

// Standalone split-precision transform (for testing the building block):
// out[r][j] = sum_k in[r][k] T[j][k], T = forward or inverse DCT matrix.
__global__ void __launch_bounds__(kTcThreads, 1) k_tc_transform(const float* in, float* out, int rows,
                                                              int n, const uint8_t* Bg) {
  extern __shared__ __align__(1024) uint8_t tc_smem_raw[];
  TcSmem* sm = reinterpret_cast<TcSmem*>(
      (reinterpret_cast<uintptr_t>(tc_smem_raw) + 1023) & ~(uintptr_t)1023);
  if (threadIdx.x == 0) {
    vstc::mbar_init(&sm->full[0], 1);
    vstc::mbar_init(&sm->full[1], 1);
    vstc::mbar_init(&sm->done[0], 1);
    vstc::mbar_init(&sm->done[1], 1);
    vstc::mbar_init(&sm->fin, 1);
    vstc::mbar_fence_init();
    sm->err = 0u;
  }
  if ((threadIdx.x >> 5) == 0) vstc::tmem_alloc(&sm->tmem_base, 256);
  vstc::tc_fence_before();
  __syncthreads();
  vstc::tc_fence_after();
  TcCtx c;
  c.sm = sm;
  c.tmem = sm->tmem_base;
  c.uses[0] = c.uses[1] = 0;
  c.chunk = 0;
  c.fin_uses = 0;
  const int NB = n < 256 ? n : 256;
  const size_t bstride = (size_t)(n / kTcChunkK) * 2 * NB * kTcChunkK * 2;
  bool ok = true;
  for (int t = blockIdx.x; t < rows / 128 && ok; t += gridDim.x) {
    for (int nc = 0; nc < n / NB && ok; ++nc) {
      ok = tc_gemm(c, n, NB, Bg + nc * bstride, in, n, t * 128, nullptr);
      if (!ok) break;
      tc_epilogue(c, NB, [&](int m, int c0, float* v) {
        store32(out + (size_t)(t * 128 + m) * n + nc * NB + c0, v);
      });
      vstc::tc_fence_before();
      __syncthreads();
    }
  }
  tc_finish(c);
}

// ------------------------------------------------------------ host side

std::vector<int> host_digrev(int n) {
  std::vector<int> rad;
  int rem = n;
  while (rem > 1) {
    int r = rem >= 16 ? 16 : rem;
    rad.push_back(r);
    rem /= r;
  }
  std::vector<int> out(n);
  for (int k = 0; k < n; ++k) {
    int kk = k, m = n, p = 0;
    for (int r : rad) {
      m /= r;
      p += (kk % r) * m;
      kk /= r;
    }
    out[k] = p;
  }
  return out;
}

std::mutex g_fft_mutex;
std::map<std::pair<int, int>, vs_fft_tables*> g_fft;

// ---- pre-split, pre-tiled DCT matrices for the tensor-core path
uint16_t host_bf16(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);          // round to nearest even
  return (uint16_t)(u >> 16);
}
double host_bf16_val(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

struct TcMats {
  uint8_t* fwd = nullptr;    // B[j][k] = cos(pi j (2k+1) / 2n)
  uint8_t* inv = nullptr;    // B[j][k] = w_k cos(pi k (2j+1) / 2n) / n
};
std::mutex g_tc_mutex;
std::map<std::pair<int, int>, TcMats> g_tc;

// Layout: for each output chunk of NB = min(n, 256) rows j and each K-chunk of
// 64 columns k: [hi: NB x 64 in core-matrix order][lo: same].
std::vector<uint8_t> tile_matrix(int n, bool inverse) {
  const double pi = 3.141592653589793238462643383279502884;
  const int nk = n / kTcChunkK;
  const int NB = n < 256 ? n : 256;
  const size_t half = (size_t)NB * kTcChunkK * 2;
  std::vector<uint8_t> out((size_t)(n / NB) * nk * 2 * half, 0);
  for (int j = 0; j < n; ++j)
    for (int k = 0; k < n; ++k) {
      double v = inverse ? (k == 0 ? 1.0 : 2.0) * cos(pi * k * (2.0 * j + 1.0) / (2.0 * n)) / n
                         : cos(pi * j * (2.0 * k + 1.0) / (2.0 * n));
      uint16_t hi = host_bf16(v);
      uint16_t lo = host_bf16(v - host_bf16_val(hi));
      int kc = k / kTcChunkK, nc = j / NB;
      size_t off = ((size_t)nc * nk + kc) * 2 * half + vstc::core_off(j % NB, k % kTcChunkK, kTcChunkK);
      memcpy(&out[off], &hi, 2);
      memcpy(&out[off + half], &lo, 2);
    }
  return out;
}

const TcMats* get_tc_mats(int n, int* status) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_tc_mutex);
  auto key = std::make_pair(dev, n);
  auto it = g_tc.find(key);
  if (it != g_tc.end()) return &it->second;
  TcMats m;
  std::vector<uint8_t> f = tile_matrix(n, false), iv = tile_matrix(n, true);
  cudaError_t e = cudaMalloc(&m.fwd, f.size());
  if (e == cudaSuccess) e = cudaMalloc(&m.inv, iv.size());
  if (e == cudaSuccess) e = cudaMemcpy(m.fwd, f.data(), f.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m.inv, iv.data(), iv.size(), cudaMemcpyHostToDevice);
  if (e != cudaSuccess) {
    cudaFree(m.fwd);
    cudaFree(m.inv);
    *status = vs_set_error(e == cudaErrorMemoryAllocation ? VS_ERR_OOM : VS_ERR_CUDA,
                           "tensor-core matrices n=%d: %s", n, cudaGetErrorString(e));
    return nullptr;
  }
  g_tc[key] = m;
  return &g_tc[key];
}

bool tc_size_ok(int n) { return n >= 128 && n <= 1024; }   // n is a power of two
constexpr size_t kTcSmemBytes = sizeof(TcSmem) + 1024;

struct TaskShape {
  int elems;   // target elements per task
};

int rows_for(int n, int elems) { return std::max(2, std::min(n, std::min(64, elems / n))); }
int cols_for(int n, int elems) { return std::max(2, std::min(n, std::min(64, elems / n))); }

}  // namespace

const vs_fft_tables* vs_get_fft_tables(int n, int* status) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_fft_mutex);
  auto key = std::make_pair(dev, n);
  auto it = g_fft.find(key);
  if (it != g_fft.end()) return it->second;
  vs_fft_tables* t = new vs_fft_tables();
  t->n = n;
  std::vector<int> dr = host_digrev(n);
  cudaError_t e = cudaMalloc(&t->tw4n, sizeof(float2) * 4 * n);
  if (e == cudaSuccess) e = cudaMalloc(&t->digrev, sizeof(int) * n);
  if (e == cudaSuccess) e = cudaMemcpy(t->digrev, dr.data(), sizeof(int) * n, cudaMemcpyHostToDevice);
  if (e == cudaSuccess) {
    k_twiddles<<<(4 * n + 255) / 256, 256>>>(n, t->tw4n);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess) e = cudaDeviceSynchronize();
  if (e != cudaSuccess) {
    cudaFree(t->tw4n);
    cudaFree(t->digrev);
    delete t;
    *status = vs_set_error(e == cudaErrorMemoryAllocation ? VS_ERR_OOM : VS_ERR_CUDA,
                           "FFT tables for n=%d: %s", n, cudaGetErrorString(e));
    return nullptr;
  }
  g_fft[key] = t;
  return t;
}

// ---------------------------------------------------------------- plans

struct vs_plan_t {
  int n_items;
  std::vector<vs_batch_item> items;
  vs_solve_params params;
  int elems;                 // task size
  int grid;
  size_t smem;
  int row_tasks, col_tasks, part_total;
  MapDesc* d_maps = nullptr;
  int* d_row_map = nullptr;
  int* d_col_map = nullptr;
  MapState* d_state = nullptr;
  double* d_part = nullptr;
  vs_solve_info* d_info = nullptr;
  Ctrl* d_ctrl = nullptr;
  float* d_work = nullptr;
  float* d_trstate = nullptr;
  int transient_steps = 0;
  int tr_window = 0;                          // transient options (vs_transient_opts)
  int tr_implicit = 0;
  int tr_slices = 1;                          // n*n slices of per-mode state per map
  int warm = 0;
  bool cluster = false;                       // cluster engine
  std::vector<std::pair<int, int>> cl_groups; // (n, maps) per launch, in order
  int* d_order = nullptr;                     // maps grouped by n
  int cl_batch = kClBatchDefault;             // cluster engine: update-load batch
  bool tcc = false;                           // split precision with the map on chip
  // autotuner record: the candidate shapes timed at creation and their times
  std::vector<std::pair<int, double>> tuned;
};

namespace {

std::mutex g_tune_mutex;
std::mutex g_attr_mutex;
size_t g_smem_attr_steady = 0, g_smem_attr_steady_phys = 0, g_smem_attr_transient = 0,
       g_smem_attr_transient_var = 0;
std::map<std::vector<int>, int> g_tuned;  // key: sorted n list + batch bucket

void plan_release(vs_plan_t* p) {
  cudaFree(p->d_maps);
  cudaFree(p->d_row_map);
  cudaFree(p->d_col_map);
  cudaFree(p->d_state);
  cudaFree(p->d_part);
  cudaFree(p->d_info);
  cudaFree(p->d_ctrl);
  cudaFree(p->d_work);
  cudaFree(p->d_trstate);
  cudaFree(p->d_order);
  p->d_order = nullptr;
  p->d_maps = nullptr;
  p->d_row_map = nullptr;
  p->d_col_map = nullptr;
  p->d_state = nullptr;
  p->d_part = nullptr;
  p->d_info = nullptr;
  p->d_ctrl = nullptr;
  p->d_work = nullptr;
  p->d_trstate = nullptr;
}

// Builds descriptors and scratch for task size `elems`.
int plan_layout(vs_plan_t* p, int elems, cudaStream_t s, bool transient, int n_steps) {
  plan_release(p);
  p->elems = elems;
  int n_items = p->n_items;
  std::vector<MapDesc> maps(n_items);
  size_t work_total = 0;
  int row_off = 0, col_off = 0, part_off = 0;
  size_t smem = 0;
  const bool tc = p->params.precision == VS_PREC_BF16_SPLIT;
  for (int i = 0; i < n_items; ++i) {
    const vs_batch_item& it = p->items[i];
    vs_kernel k = it.k;
    int n = k->n;
    MapDesc& m = maps[i];
    if (tc) {
      int st = VS_OK;
      const TcMats* tm = get_tc_mats(n, &st);
      if (!tm) return st;
      m.tcf = tm->fwd;
      m.tci = tm->inv;
    }
    m.p_dyn = it.p_dyn;
    m.p_leak0 = it.p_leak0;
    m.s = it.s_kappa;
    m.theta = it.theta;
    m.theta_init = it.theta_init;
    if (it.theta_init) p->warm = 1;
    m.Kt = k->Kt32;
    m.tw4n = k->fft->tw4n;
    m.digrev = k->fft->digrev;
    m.trA = k->trA;
    m.trRho = k->trRho;
    m.kmax = k->kmax;
    m.n = n;
    m.rb = tc ? 128 : rows_for(n, elems);
    m.cb = tc ? 128 : cols_for(n, elems);
    m.row_off = row_off;
    m.col_off = col_off;
    m.part_off = part_off;
    row_off += n / m.rb;
    col_off += n / m.cb;
    part_off += n / m.rb;
    work_total += (size_t)n * n * (tc ? 2 : 1);
    size_t sm = tc ? kTcSmemBytes : (size_t)(std::max(m.rb, m.cb) / 2) * padded_len(n) * sizeof(float2);
    smem = std::max(smem, sm);
  }
  p->row_tasks = row_off;
  p->col_tasks = col_off;
  p->part_total = part_off;
  p->smem = smem;
  VS_CUDA_TRY(cudaMalloc(&p->d_work, work_total * sizeof(float)));
  if (transient)
    VS_CUDA_TRY(cudaMalloc(&p->d_trstate, work_total * (size_t)p->tr_slices * sizeof(float)));
  size_t off = 0;
  for (int i = 0; i < n_items; ++i) {
    maps[i].work = p->d_work + off;
    maps[i].state = transient ? p->d_trstate + off * p->tr_slices : nullptr;
    off += (size_t)maps[i].n * maps[i].n;
    if (tc) {
      maps[i].work2 = p->d_work + off;
      off += (size_t)maps[i].n * maps[i].n;
    }
  }
  VS_CUDA_TRY(cudaMalloc(&p->d_maps, sizeof(MapDesc) * n_items));
  VS_CUDA_TRY(cudaMalloc(&p->d_state, sizeof(MapState) * n_items));
  VS_CUDA_TRY(cudaMalloc(&p->d_part, 2 * sizeof(double) * std::max(1, part_off)));   // part, part2
  VS_CUDA_TRY(cudaMalloc(&p->d_info, sizeof(vs_solve_info) * n_items));
  VS_CUDA_TRY(cudaMalloc(&p->d_ctrl, sizeof(Ctrl)));
  VS_CUDA_TRY(cudaMemcpyAsync(p->d_maps, maps.data(), sizeof(MapDesc) * n_items,
                              cudaMemcpyHostToDevice, s));
  std::vector<int> rmap(p->row_tasks), cmap(p->col_tasks);
  for (int i = 0; i < n_items; ++i) {
    for (int t = 0; t < maps[i].n / maps[i].rb; ++t) rmap[maps[i].row_off + t] = i;
    for (int t = 0; t < maps[i].n / maps[i].cb; ++t) cmap[maps[i].col_off + t] = i;
  }
  VS_CUDA_TRY(cudaMalloc(&p->d_row_map, sizeof(int) * p->row_tasks));
  VS_CUDA_TRY(cudaMalloc(&p->d_col_map, sizeof(int) * p->col_tasks));
  VS_CUDA_TRY(cudaMemcpyAsync(p->d_row_map, rmap.data(), sizeof(int) * p->row_tasks,
                              cudaMemcpyHostToDevice, s));
  VS_CUDA_TRY(cudaMemcpyAsync(p->d_col_map, cmap.data(), sizeof(int) * p->col_tasks,
                              cudaMemcpyHostToDevice, s));
  VS_CUDA_TRY(cudaMemsetAsync(p->d_info, 0, sizeof(vs_solve_info) * n_items, s));

  const bool tr_var = transient && (p->tr_window || p->tr_implicit);
  auto fn = tr_var    ? (const void*)k_solve_transient_var
            : transient ? (const void*)k_solve_transient
            : tc      ? (const void*)k_solve_steady_tc
                      : vs_params_physics(&p->params) ? (const void*)k_solve_steady<true>
                                                      : (const void*)k_solve_steady<false>;
  if (tc) {
    VS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
    VS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  } else {
    // Function attributes are process-wide: only ever raise the limit, so a
    // plan with a smaller footprint never invalidates a larger one.
    std::lock_guard<std::mutex> lk(g_attr_mutex);
    size_t& cur = tr_var ? g_smem_attr_transient_var
                  : transient ? g_smem_attr_transient
                  : vs_params_physics(&p->params) ? g_smem_attr_steady_phys : g_smem_attr_steady;
    if (smem > cur) {
      VS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      VS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
      cur = smem;
    }
  }
  int per_sm = 0;
  VS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, fn, tc ? kTcThreads : kThreads,
                                                            smem));
  if (per_sm < 1) return vs_set_error(VS_ERR_INVALID_ARG, "no block fits on an SM (smem %zu)", smem);
  int dev = 0, sms = 0;
  VS_CUDA_TRY(cudaGetDevice(&dev));
  VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int want = std::max(p->row_tasks, p->col_tasks);
  p->grid = std::max(1, std::min(per_sm * sms, want));
  if (getenv("VS_DEBUG")) {
    cudaFuncAttributes fa;
    cudaFuncGetAttributes(&fa, fn);
    int smem_sm = 0, regs_sm = 0;
    cudaDeviceGetAttribute(&smem_sm, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    cudaDeviceGetAttribute(&regs_sm, cudaDevAttrMaxRegistersPerMultiprocessor, dev);
    fprintf(stderr,
            "varsim plan: %s items=%d grid=%d per_sm=%d sms=%d smem=%zu tasks=%d/%d regs=%d "
            "static_smem=%zu max_dyn=%d local=%zu | sm: smem=%d regs=%d\n",
            transient ? "transient" : (tc ? "bf16-split" : "fp32"), n_items, p->grid, per_sm, sms,
            smem, p->row_tasks, p->col_tasks, fa.numRegs, fa.sharedSizeBytes,
            fa.maxDynamicSharedSizeBytes, fa.localSizeBytes, smem_sm, regs_sm);
  }
  p->transient_steps = n_steps;
  VS_CUDA_TRY(cudaStreamSynchronize(s));  // host `maps` must outlive the copy
  return VS_OK;
}

size_t g_smem_attr_cluster[4][3] = {};  // per instantiation: n = 32 .. 256 x batch 1, 2, 4

int batch_index(int b) { return b == 1 ? 0 : b == 4 ? 2 : 1; }

// Shared-memory attributes of the cluster instantiation (n, batch), once.
int cluster_attrs(int n, int batch) {
  std::lock_guard<std::mutex> lk(g_attr_mutex);
  size_t& cur = g_smem_attr_cluster[__builtin_ctz((unsigned)n) - 5][batch_index(batch)];
  if (cur == 0) {
    ClusterFn fn = cluster_kernel(n, batch);
    VS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cluster_shape(n).smem));
    VS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    cur = cluster_shape(n).smem;
  }
  return VS_OK;
}

// Shared-memory attributes of the physics-variant instantiation for n, once.
int cluster_attrs_phys(int n) {
  static size_t done[4] = {};
  std::lock_guard<std::mutex> lk(g_attr_mutex);
  size_t& cur = done[__builtin_ctz((unsigned)n) - 5];
  if (cur == 0) {
    ClusterFn fn = cluster_kernel_phys(n);
    VS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)cluster_shape(n).smem));
    VS_CUDA_TRY(cudaFuncSetAttribute(fn, cudaFuncAttributePreferredSharedMemoryCarveout, 100));
    cur = cluster_shape(n).smem;
  }
  return VS_OK;
}

cudaLaunchConfig_t cluster_config(int n, int count, cudaStream_t s, cudaLaunchAttribute* attr) {
  cudaLaunchConfig_t cfg = {};
  const ClHost h = cluster_shape(n);
  cfg.gridDim = dim3((unsigned)h.ranks * (unsigned)count);
  cfg.blockDim = dim3((unsigned)h.threads);
  cfg.dynamicSmemBytes = h.smem;
  cfg.stream = s;
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = (unsigned)h.ranks;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  return cfg;
}

// Cluster engine layout: descriptors only (no spectral scratch), maps grouped
// by grid size, one launch per group.
int plan_layout_cluster(vs_plan_t* p, cudaStream_t s) {
  plan_release(p);
  const int n_items = p->n_items;
  std::map<int, std::vector<int>> by_n;
  for (int i = 0; i < n_items; ++i) by_n[p->items[i].k->n].push_back(i);
  std::vector<int> order;
  p->cl_groups.clear();
  size_t smem = 0;
  for (auto& g : by_n) {
    p->cl_groups.push_back({g.first, (int)g.second.size()});
    order.insert(order.end(), g.second.begin(), g.second.end());
    smem = std::max(smem, cluster_shape(g.first).smem);
  }
  std::vector<MapDesc> maps(n_items);
  for (int i = 0; i < n_items; ++i) {
    const vs_batch_item& it = p->items[i];
    MapDesc& m = maps[i];
    memset(&m, 0, sizeof(m));
    m.p_dyn = it.p_dyn;
    m.p_leak0 = it.p_leak0;
    m.s = it.s_kappa;
    m.theta = it.theta;
    m.theta_init = it.theta_init;
    if (it.theta_init) p->warm = 1;
    m.Kt = it.k->Kt32;
    m.tw4n = it.k->fft->tw4n;
    m.digrev = it.k->fft->digrev;
    m.kmax = it.k->kmax;
    m.n = it.k->n;
  }
  p->smem = smem;
  VS_CUDA_TRY(cudaMalloc(&p->d_maps, sizeof(MapDesc) * n_items));
  VS_CUDA_TRY(cudaMalloc(&p->d_order, sizeof(int) * n_items));
  VS_CUDA_TRY(cudaMalloc(&p->d_info, sizeof(vs_solve_info) * n_items));
  VS_CUDA_TRY(cudaMalloc(&p->d_ctrl, sizeof(Ctrl)));
  VS_CUDA_TRY(cudaMemcpyAsync(p->d_maps, maps.data(), sizeof(MapDesc) * n_items,
                              cudaMemcpyHostToDevice, s));
  VS_CUDA_TRY(cudaMemcpyAsync(p->d_order, order.data(), sizeof(int) * n_items,
                              cudaMemcpyHostToDevice, s));
  VS_CUDA_TRY(cudaMemsetAsync(p->d_info, 0, sizeof(vs_solve_info) * n_items, s));
  VS_CUDA_TRY(cudaMemsetAsync(p->d_ctrl, 0, sizeof(Ctrl), s));
  if (p->tcc) {
    int rc = vs_tcc_check(s);
    if (rc != VS_OK) return rc;
    p->grid = 0;
    VS_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors must outlive the copies
    return VS_OK;
  }
  for (auto& g : p->cl_groups) {
    ClusterFn fn = cluster_kernel(g.first, p->cl_batch);
    int rc = cluster_attrs(g.first, p->cl_batch);
    if (rc != VS_OK) return rc;
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(g.first, 1, s, attr);
    int clusters = 0;
    VS_CUDA_TRY(cudaOccupancyMaxActiveClusters(&clusters, fn, &cfg));
    if (clusters < 1)
      return vs_set_error(VS_ERR_INVALID_ARG, "no cluster of %d CTAs fits on the device (n=%d)",
                          cluster_shape(g.first).ranks, g.first);
    if (getenv("VS_DEBUG")) {
      cudaFuncAttributes fa;
      cudaFuncGetAttributes(&fa, fn);
      fprintf(stderr, "varsim plan: cluster n=%d maps=%d ranks=%d smem=%zu regs=%d local=%zu "
              "active_clusters=%d\n", g.first, g.second, cluster_shape(g.first).ranks, cluster_shape(g.first).smem,
              fa.numRegs, fa.localSizeBytes, clusters);
    }
  }
  p->grid = 0;
  VS_CUDA_TRY(cudaStreamSynchronize(s));  // host vectors must outlive the copies
  return VS_OK;
}

int plan_launch_cluster(vs_plan_t* p, cudaStream_t s) {
  int off = 0;
  for (auto& g : p->cl_groups) {
    ClusterDev P;
    P.maps = p->d_maps;
    P.order = p->d_order + off;
    P.info = p->d_info;
    P.max_iter = p->params.max_iter;
    P.beta = (float)p->params.beta_per_K;
    P.alpha = (float)p->params.alpha_per_K;
    P.tol = (float)p->params.tol_K;
    P.stop_rule = p->params.stop_rule;
    if (p->tcc) {
      int rc = vs_tcc_launch(P, g.second, s);
      if (rc != VS_OK) return rc;
      off += g.second;
      continue;
    }
    const vs_solve_params& pp = p->params;
    const bool phys = vs_params_physics(&pp) != 0;
    if (phys) {
      P.cond = pp.conductivity;
      P.one_me = (float)(1.0 - pp.eta);
      P.t_amb = (float)pp.t_amb_K;
      P.leak_n = pp.leak_points;
      for (int i = 0; i < VS_MAX_LEAK_POINTS; ++i) {
        P.leak_x[i] = i < pp.leak_points ? (float)pp.leak_theta_K[i] : 0.f;
        P.leak_y[i] = i < pp.leak_points ? (float)pp.leak_g[i] : 0.f;
      }
      if (pp.leak_points >= 2) {
        // precondition with the slope of the table at theta = 0, as the streamed engine
        int i = 0;
        while (i < pp.leak_points - 2 && pp.leak_theta_K[i + 1] <= 0.0) ++i;
        P.beta = (float)std::max(0.0, (pp.leak_g[i + 1] - pp.leak_g[i]) /
                                          (pp.leak_theta_K[i + 1] - pp.leak_theta_K[i]));
      }
      int rc = cluster_attrs_phys(g.first);
      if (rc != VS_OK) return rc;
    }
    cudaLaunchAttribute attr[1];
    cudaLaunchConfig_t cfg = cluster_config(g.first, g.second, s, attr);
    cudaError_t e = cudaLaunchKernelEx(
        &cfg, phys ? cluster_kernel_phys(g.first) : cluster_kernel(g.first, p->cl_batch), P);
    if (e != cudaSuccess)
      return vs_set_error(VS_ERR_CUDA, "cluster launch (n %d, %d maps): %s", g.first, g.second,
                          cudaGetErrorString(e));
    off += g.second;
  }
  return VS_OK;
}

int plan_launch(vs_plan_t* p, cudaStream_t s, bool transient) {
  if (p->cluster && !transient) return plan_launch_cluster(p, s);
  VS_CUDA_TRY(cudaMemsetAsync(p->d_ctrl, 0, sizeof(Ctrl), s));
  VS_CUDA_TRY(cudaMemsetAsync(p->d_state, 0, sizeof(MapState) * p->n_items, s));
  PlanDev P = {};
  P.maps = p->d_maps;
  P.row_map = p->d_row_map;
  P.col_map = p->d_col_map;
  P.st = p->d_state;
  P.part = p->d_part;
  P.part2 = p->d_part + std::max(1, p->part_total);
  P.info = p->d_info;
  P.ctrl = p->d_ctrl;
  P.n_maps = p->n_items;
  P.row_tasks = p->row_tasks;
  P.col_tasks = p->col_tasks;
  P.max_iter = p->params.max_iter;
  P.beta = (float)p->params.beta_per_K;
  P.alpha = (float)p->params.alpha_per_K;
  P.tol = (float)p->params.tol_K;
  P.stop_rule = p->params.stop_rule;
  P.n_steps = p->transient_steps;
  P.warm = p->warm;
  const vs_solve_params& pp = p->params;
  P.cond = pp.conductivity;
  P.one_me = (float)(1.0 - pp.eta);
  P.t_amb = (float)pp.t_amb_K;
  P.leak_n = pp.leak_points;
  for (int i = 0; i < VS_MAX_LEAK_POINTS; ++i) {
    P.leak_x[i] = i < pp.leak_points ? (float)pp.leak_theta_K[i] : 0.f;
    P.leak_y[i] = i < pp.leak_points ? (float)pp.leak_g[i] : 0.f;
  }
  if (pp.leak_points >= 2) {
    // precondition with the slope of the table at theta = 0 (any slope gives
    // the same fixed point; it also sets the runaway check beta mu max K < 1)
    int i = 0;
    while (i < pp.leak_points - 2 && pp.leak_theta_K[i + 1] <= 0.0) ++i;
    P.beta = (float)std::max(0.0, (pp.leak_g[i + 1] - pp.leak_g[i]) /
                                      (pp.leak_theta_K[i + 1] - pp.leak_theta_K[i]));
  }
  P.adaptive = !transient && pp.precision == VS_PREC_FP32 && !vs_params_physics(&pp);
  P.window = transient ? p->tr_window : 0;
  P.implicit = transient ? p->tr_implicit : 0;
  // the implicit transient keeps the current step's source spectrum in the
  // last state slice (one map per transient plan)
  P.xs = (transient && p->tr_implicit)
             ? p->d_trstate + (size_t)(p->tr_slices - 1) * p->items[0].k->n * p->items[0].k->n
             : nullptr;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(p->grid);
  cfg.blockDim = dim3(p->params.precision == VS_PREC_BF16_SPLIT && !transient ? kTcThreads : kThreads);
  cfg.dynamicSmemBytes = p->smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = transient ? ((P.window || P.implicit) ? cudaLaunchKernelEx(&cfg, k_solve_transient_var, P)
                                                       : cudaLaunchKernelEx(&cfg, k_solve_transient, P))
                  : p->params.precision == VS_PREC_BF16_SPLIT
                      ? cudaLaunchKernelEx(&cfg, k_solve_steady_tc, P)
                  : vs_params_physics(&p->params) ? cudaLaunchKernelEx(&cfg, k_solve_steady<true>, P)
                                                  : cudaLaunchKernelEx(&cfg, k_solve_steady<false>, P);
  if (e != cudaSuccess)
    return vs_set_error(VS_ERR_CUDA, "cooperative launch (grid %d, smem %zu): %s", p->grid,
                        p->smem, cudaGetErrorString(e));
  return VS_OK;
}

int timeout_status(vs_plan_t* p, cudaStream_t s) {
  Ctrl c;
  VS_CUDA_TRY(cudaMemcpyAsync(&c, p->d_ctrl, sizeof(unsigned) * 4, cudaMemcpyDeviceToHost, s));
  VS_CUDA_TRY(cudaStreamSynchronize(s));
  if (c.abort) return vs_set_error(VS_ERR_TIMEOUT, "grid barrier timed out");
  return VS_OK;
}

double time_plan(vs_plan_t* p, cudaStream_t s, int reps) {
  cudaEvent_t a, b;
  cudaEventCreate(&a);
  cudaEventCreate(&b);
  if (plan_launch(p, s, false) != VS_OK) return 1e30;
  cudaEventRecord(a, s);
  for (int i = 0; i < reps; ++i)
    if (plan_launch(p, s, false) != VS_OK) return 1e30;
  cudaEventRecord(b, s);
  cudaEventSynchronize(b);
  float ms = 0.f;
  cudaEventElapsedTime(&ms, a, b);
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms;
}

}  // namespace

// ---------------------------------------------------------------------------
// Autotuner of the launch shape. A plan's shape is one integer: the cluster
// engine's update-load batch (1, 2 or 4 positions whose inputs a thread loads
// before using them), or the streamed engine's task size (elements of a map per
// row/column task: 2048, 4096, 8192 or 16384). Plans of at least 64 maps are
// tuned by timing every candidate on the plan itself (one warm-up and two timed
// runs each, CUDA events) and keeping the fastest; the choice is cached per
// engine, mix of grid sizes and batch size (power-of-two bucket), so later
// plans of the same kind are not timed again. VS_AUTOTUNE=0 keeps the defaults.
// ---------------------------------------------------------------------------
namespace {

std::vector<int> tune_key(const vs_batch_item* items, int n_items, bool cluster) {
  std::vector<int> key;
  for (int i = 0; i < n_items; ++i) key.push_back(items[i].k->n);
  std::sort(key.begin(), key.end());
  key.erase(std::unique(key.begin(), key.end()), key.end());
  int bucket = 0;
  while ((1 << (bucket + 1)) <= n_items) ++bucket;
  key.push_back(bucket);
  key.push_back(cluster ? 1 : 0);
  return key;
}

bool tune_enabled(int n_items) {
  const char* env = getenv("VS_AUTOTUNE");
  return n_items >= 64 && !(env && env[0] == '0');
}

bool cluster_shape_ok(int b) { return b == 1 || b == 2 || b == 4; }
bool streamed_shape_ok(int e) { return e == 2048 || e == 4096 || e == 8192 || e == 16384; }

}  // namespace

// shape: > 0 forced; 0 the cached choice, else tuned on the plan; -1 the
// cached choice, else the default, never timed (for plans whose buffers do
// not hold their maps yet)
int plan_create(const vs_batch_item* items_host, int n_items, const vs_solve_params* params,
                int shape, vs_plan* out, void* stream);

extern "C" int vs_plan_create(const vs_batch_item* items_host, int n_items,
                              const vs_solve_params* params, vs_plan* out, void* stream) {
  return plan_create(items_host, n_items, params, 0, out, stream);
}

extern "C" int vs_plan_create_shaped(const vs_batch_item* items_host, int n_items,
                                     const vs_solve_params* params, int shape, vs_plan* out,
                                     void* stream) {
  if (shape < 0) return vs_set_error(VS_ERR_INVALID_ARG, "shape %d", shape);
  return plan_create(items_host, n_items, params, shape, out, stream);
}

extern "C" int vs_plan_shape(vs_plan p, int* shape_out, int* n_timed, int* cand_shapes,
                             double* cand_ms) {
  if (!p) return vs_set_error(VS_ERR_INVALID_ARG, "NULL plan");
  if (shape_out) *shape_out = p->cluster ? p->cl_batch : p->elems;
  if (n_timed) *n_timed = (int)p->tuned.size();
  for (size_t i = 0; i < p->tuned.size(); ++i) {
    if (cand_shapes) cand_shapes[i] = p->tuned[i].first;
    if (cand_ms) cand_ms[i] = p->tuned[i].second;
  }
  return VS_OK;
}

int plan_create(const vs_batch_item* items_host, int n_items, const vs_solve_params* params,
                int shape, vs_plan* out, void* stream) {
  if (!out) return vs_set_error(VS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!items_host || n_items <= 0) return vs_set_error(VS_ERR_INVALID_ARG, "no items");
  int rc = vs_validate_params(params);
  if (rc) return rc;
  for (int i = 0; i < n_items; ++i) {
    const vs_batch_item& it = items_host[i];
    if (!it.k || !it.p_dyn || !it.p_leak0 || !it.theta)
      return vs_set_error(VS_ERR_INVALID_ARG, "item %d has a NULL kernel or map", i);
    uintptr_t al = (uintptr_t)it.p_dyn | (uintptr_t)it.p_leak0 | (uintptr_t)it.theta |
                   (uintptr_t)it.s_kappa | (uintptr_t)it.theta_init;
    if (al & 15u) return vs_set_error(VS_ERR_INVALID_ARG, "item %d: maps must be 16-byte aligned", i);
    if (params->precision == VS_PREC_BF16_SPLIT && !tc_size_ok(it.k->n))
      return vs_set_error(VS_ERR_INVALID_ARG,
                          "item %d: the BF16 split tensor-core path supports n = 128 .. 1024 (got %d)",
                          i, it.k->n);
  }
  if (vs_params_physics(params) && params->precision != VS_PREC_FP32)
    return vs_set_error(VS_ERR_INVALID_ARG, "the physics variants need FP32 precision");
  bool cluster_ok = params->precision == VS_PREC_FP32;
  for (int i = 0; i < n_items && cluster_ok; ++i) cluster_ok = cluster_size_ok(items_host[i].k->n);
  if (params->engine == VS_ENGINE_CLUSTER && params->precision == VS_PREC_FP32 && !cluster_ok)
    return vs_set_error(VS_ERR_INVALID_ARG,
                        "the cluster engine needs FP32 precision and every n in [32, %d]", kClMaxN);
  // split precision: the on-chip pair engine for n = 256 cold starts (engine
  // AUTO or CLUSTER), the streamed tensor-core engine otherwise (STREAMED)
  bool tcc_ok = params->precision == VS_PREC_BF16_SPLIT && !vs_params_physics(params);
  for (int i = 0; i < n_items && tcc_ok; ++i)
    tcc_ok = vs_tcc_ok(items_host[i].k->n) && !items_host[i].theta_init;
  if (params->precision == VS_PREC_BF16_SPLIT && params->engine == VS_ENGINE_CLUSTER && !tcc_ok)
    return vs_set_error(VS_ERR_INVALID_ARG,
                        "the split-precision cluster engine needs n = 256 and cold starts");
  cudaStream_t s = (cudaStream_t)stream;
  vs_plan_t* p = new vs_plan_t();
  p->n_items = n_items;
  p->items.assign(items_host, items_host + n_items);
  p->params = *params;
  if (tcc_ok && params->engine != VS_ENGINE_STREAMED) {
    if (shape > 0) {
      delete p;
      return vs_set_error(VS_ERR_INVALID_ARG, "the split-precision cluster engine has one shape (0)");
    }
    p->cluster = true;
    p->tcc = true;
    rc = plan_layout_cluster(p, s);
    if (rc != VS_OK) {
      plan_release(p);
      delete p;
      return rc;
    }
    *out = p;
    return VS_OK;
  }
  if (cluster_ok && params->engine != VS_ENGINE_STREAMED) {
    p->cluster = true;
    if (shape > 0 && !cluster_shape_ok(shape)) {
      delete p;
      return vs_set_error(VS_ERR_INVALID_ARG, "cluster engine shape %d (update batch 1, 2 or 4)",
                          shape);
    }
    const std::vector<int> key = tune_key(items_host, n_items, true);
    // the physics variants have one instantiation (update-load batch 2)
    const bool phys = vs_params_physics(params) != 0;
    if (phys && shape > 0 && shape != kClBatchDefault) {
      delete p;
      return vs_set_error(VS_ERR_INVALID_ARG,
                          "the physics variants on the cluster engine have one shape (%d)",
                          kClBatchDefault);
    }
    bool tune = shape == 0 && tune_enabled(n_items) && !phys;
    p->cl_batch = shape > 0 ? shape : kClBatchDefault;
    if (shape <= 0 && tune_enabled(n_items) && !phys) {
      std::lock_guard<std::mutex> lk(g_tune_mutex);
      auto itc = g_tuned.find(key);
      if (itc != g_tuned.end()) {
        p->cl_batch = itc->second;
        tune = false;
      }
    }
    rc = plan_layout_cluster(p, s);
    if (rc == VS_OK && tune) {
      double best = 1e30;
      int best_b = p->cl_batch;
      for (int b : kClBatches) {
        p->cl_batch = b;
        for (auto& g : p->cl_groups)
          if (rc == VS_OK) rc = cluster_attrs(g.first, b);
        if (rc != VS_OK) break;
        const double t = time_plan(p, s, 2);
        p->tuned.push_back({b, t});
        if (t < best) {
          best = t;
          best_b = b;
        }
      }
      p->cl_batch = best_b;
      if (rc == VS_OK && best < 1e29) {
        std::lock_guard<std::mutex> lk(g_tune_mutex);
        g_tuned[key] = best_b;
      }
      cudaError_t e = cudaStreamSynchronize(s);
      if (e != cudaSuccess && rc == VS_OK)
        rc = vs_set_error(VS_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
    }
    if (rc != VS_OK) {
      plan_release(p);
      delete p;
      return rc;
    }
    *out = p;
    return VS_OK;
  }

  // task size of the streamed engine: forced, cached, tuned, or the default
  if (shape > 0 && !streamed_shape_ok(shape)) {
    delete p;
    return vs_set_error(VS_ERR_INVALID_ARG,
                        "streamed engine shape %d (task size 2048, 4096, 8192 or 16384)", shape);
  }
  const std::vector<int> key = tune_key(items_host, n_items, false);
  int elems = shape > 0 ? shape : 8192;
  bool tune = shape == 0 && tune_enabled(n_items) && params->precision == VS_PREC_FP32;
  if (shape <= 0 && tune_enabled(n_items) && params->precision == VS_PREC_FP32) {
    std::lock_guard<std::mutex> lk(g_tune_mutex);
    auto itc = g_tuned.find(key);
    if (itc != g_tuned.end()) {
      elems = itc->second;
      tune = false;
    }
  }
  if (tune) {
    double best = 1e30;
    int best_e = elems;
    const int cands[4] = {2048, 4096, 8192, 16384};
    for (int e : cands) {
      rc = plan_layout(p, e, s, false, 0);
      if (rc) break;
      const double t = time_plan(p, s, 2);
      p->tuned.push_back({e, t});
      if (t < best) {
        best = t;
        best_e = e;
      }
    }
    if (rc == VS_OK && best < 1e29) {
      elems = best_e;
      std::lock_guard<std::mutex> lk(g_tune_mutex);
      g_tuned[key] = elems;
    }
    cudaError_t e = cudaStreamSynchronize(s);
    if (e != cudaSuccess && rc == VS_OK)
      rc = vs_set_error(VS_ERR_CUDA, "autotune: %s", cudaGetErrorString(e));
  }
  if (rc == VS_OK) rc = plan_layout(p, elems, s, false, 0);
  if (rc != VS_OK) {
    plan_release(p);
    delete p;
    return rc;
  }
  *out = p;
  return VS_OK;
}

extern "C" int vs_plan_run(vs_plan p, void* stream) {
  if (!p) return vs_set_error(VS_ERR_INVALID_ARG, "NULL plan");
  return plan_launch(p, (cudaStream_t)stream, false);
}

extern "C" int vs_plan_launches(vs_plan p) {
  if (!p) return 0;
  return p->cluster ? (int)p->cl_groups.size() : 1;
}

extern "C" int vs_plan_info(vs_plan p, vs_solve_info* info_host, void* stream) {
  if (!p || !info_host) return vs_set_error(VS_ERR_INVALID_ARG, "NULL plan or output");
  cudaStream_t s = (cudaStream_t)stream;
  VS_CUDA_TRY(cudaMemcpyAsync(info_host, p->d_info, sizeof(vs_solve_info) * p->n_items,
                              cudaMemcpyDeviceToHost, s));
  VS_CUDA_TRY(cudaStreamSynchronize(s));
  int rc = timeout_status(p, s);
  if (rc) return rc;
  int worst = VS_OK;
  for (int i = 0; i < p->n_items; ++i) worst = std::max(worst, info_host[i].status);
  return worst;
}

// Asynchronous copy of a plan's per-map outcome (no synchronisation, no
// timeout check), for the pipelined host-memory solve.
int vs_plan_info_async(vs_plan p, vs_solve_info* info_host, cudaStream_t s) {
  VS_CUDA_TRY(cudaMemcpyAsync(info_host, p->d_info, sizeof(vs_solve_info) * p->n_items,
                              cudaMemcpyDeviceToHost, s));
  return VS_OK;
}

// VS_ERR_TIMEOUT if the last run of the plan aborted on a barrier timeout.
int vs_plan_check_timeout(vs_plan p, cudaStream_t s) {
  return p->cluster ? VS_OK : timeout_status(p, s);
}

extern "C" void vs_plan_free(vs_plan p) {
  if (!p) return;
  plan_release(p);
  delete p;
}

extern "C" int vs_solve_batch(const vs_batch_item* items_host, int n_items,
                              const vs_solve_params* params, vs_solve_info* info_host,
                              void* stream) {
  vs_plan p = nullptr;
  int rc = vs_plan_create(items_host, n_items, params, &p, stream);
  if (rc) return rc;
  rc = vs_plan_run(p, stream);
  if (rc == VS_OK) {
    std::vector<vs_solve_info> tmp(n_items);
    rc = vs_plan_info(p, info_host ? info_host : tmp.data(), stream);
  }
  cudaStreamSynchronize((cudaStream_t)stream);
  vs_plan_free(p);
  return rc;
}

extern "C" int vs_solve_steady(vs_kernel k, const float* p_dyn, const float* p_leak0,
                               const float* s_kappa, const vs_solve_params* params, float* theta,
                               vs_solve_info* info_host, void* stream) {
  if (!k) return vs_set_error(VS_ERR_INVALID_ARG, "NULL kernel");
  vs_batch_item it = {k, p_dyn, p_leak0, s_kappa, theta, nullptr};
  vs_solve_info inf;
  int rc = vs_solve_batch(&it, 1, params, &inf, stream);
  if (info_host && (rc == VS_OK || rc >= VS_ERR_NO_CONVERGENCE)) *info_host = inf;
  return rc;
}

extern "C" int vs_solve_transient_ex(vs_kernel k, int n_steps, const float* p_dyn_trace,
                                     const float* p_leak0, const float* s_kappa,
                                     const vs_solve_params* params, const vs_transient_opts* opts,
                                     float* theta_trace, vs_solve_info* info_host, void* stream) {
  if (!k) return vs_set_error(VS_ERR_INVALID_ARG, "NULL kernel");
  if (!(k->dt > 0.0) || !k->trA)
    return vs_set_error(VS_ERR_INVALID_ARG, "kernel was built without a time step (dt_s = 0)");
  if (n_steps < 1 || n_steps > 1000000) return vs_set_error(VS_ERR_INVALID_ARG, "n_steps %d", n_steps);
  int rc = vs_validate_params(params);
  if (rc) return rc;
  if (vs_params_physics(params))
    return vs_set_error(VS_ERR_INVALID_ARG, "the transient runs the linear models only");
  const vs_transient_opts o = opts ? *opts : vs_transient_opts{0, VS_LEAK_LAGGED};
  if (o.window < 0 || o.window > VS_MAX_WINDOW)
    return vs_set_error(VS_ERR_INVALID_ARG, "window %d not in 0..%d", o.window, VS_MAX_WINDOW);
  if (o.leakage != VS_LEAK_LAGGED && o.leakage != VS_LEAK_IMPLICIT)
    return vs_set_error(VS_ERR_INVALID_ARG, "leakage mode %d", o.leakage);
  if (!p_dyn_trace || !p_leak0 || !theta_trace)
    return vs_set_error(VS_ERR_INVALID_ARG, "NULL map");
  uintptr_t al = (uintptr_t)p_dyn_trace | (uintptr_t)p_leak0 | (uintptr_t)theta_trace |
                 (uintptr_t)s_kappa;
  if (al & 15u) return vs_set_error(VS_ERR_INVALID_ARG, "maps must be 16-byte aligned");
  cudaStream_t s = (cudaStream_t)stream;
  if ((o.window == 0 || o.leakage == VS_LEAK_LAGGED) && vs_transient_fast_ok(k->n)) {
    // the persistent single-map engine (vs_transient.cu): lagged leakage with or
    // without a window, or implicit leakage without one
    vs_solve_info inf = {};
    const int r = vs_transient_fast(k, n_steps, p_dyn_trace, p_leak0, s_kappa, params,
                                    o.leakage == VS_LEAK_IMPLICIT, o.window, theta_trace, &inf, s);
    if (r != -1) {
      if (info_host && (r == VS_OK || r >= VS_ERR_NO_CONVERGENCE)) *info_host = inf;
      return r;
    }
  }
  vs_plan_t* p = new vs_plan_t();
  p->n_items = 1;
  p->items.push_back(vs_batch_item{k, p_dyn_trace, p_leak0, s_kappa, theta_trace, nullptr});
  p->params = *params;
  p->tr_window = o.window;
  p->tr_implicit = o.leakage == VS_LEAK_IMPLICIT;
  // per-mode history: the recursion state W (untruncated) or a ring of the
  // last window - 1 source spectra; plus the current source (implicit)
  p->tr_slices = std::max(1, o.window == 0 ? 1 : o.window - 1) + p->tr_implicit;
  // a single map: tasks of 4096 elements (4 rows at 1024^2) spread it over more
  // CTAs than the 8192 of batched plans (measured 46 vs 57 us per 1024^2 step)
  rc = plan_layout(p, 4096, s, true, n_steps);
  if (rc == VS_OK) {
    cudaError_t e = cudaMemsetAsync(p->d_trstate, 0,
                                    sizeof(float) * (size_t)k->n * k->n * p->tr_slices, s);
    if (e != cudaSuccess) rc = vs_set_error(VS_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
  }
  if (rc == VS_OK) rc = plan_launch(p, s, true);
  if (rc == VS_OK) {
    vs_solve_info inf;
    rc = vs_plan_info(p, &inf, stream);
    if (info_host) *info_host = inf;
  }
  cudaStreamSynchronize(s);
  plan_release(p);
  delete p;
  return rc;
}

extern "C" int vs_solve_transient(vs_kernel k, int n_steps, const float* p_dyn_trace,
                                  const float* p_leak0, const float* s_kappa,
                                  const vs_solve_params* params, float* theta_trace,
                                  vs_solve_info* info_host, void* stream) {
  return vs_solve_transient_ex(k, n_steps, p_dyn_trace, p_leak0, s_kappa, params, nullptr,
                               theta_trace, info_host, stream);
}

// ---------------------------------------------------------------------------
// Allocation-free steady solve.
//
// Some callers cannot allocate device memory at solve time: services that
// reserve their whole device-memory budget up front and forbid later
// allocations, and latency-critical loops that must not hit cudaMalloc /
// cudaFree (both can synchronise the device and take locks). For them this
// entry point keeps all per-call scratch of the steady solve (the spectral
// work map, descriptors, per-map state, reduction slots, barrier words) in one
// file-scope device array of fixed size, reserved when the library is loaded
// and held by every GPU that loads it until the process exits.
//
// The array is shared by every call: its contents persist from the previous
// call, so each call re-initialises the parts that must start at zero, and two
// calls whose work overlaps on the GPU (different streams, or different host
// threads) race on it. Calls on one stream are ordered and safe.
// ---------------------------------------------------------------------------
namespace {

constexpr int kNoAllocMaxN = 512;
constexpr size_t kNoAllocWorkBytes = (size_t)kNoAllocMaxN * kNoAllocMaxN * sizeof(float);
constexpr size_t kNoAllocBytes = kNoAllocWorkBytes + (16u << 10);

static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

struct NoAllocLayout {
  size_t desc, state, part, info, ctrl, row_map, col_map, end;
};

constexpr size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }

NoAllocLayout noalloc_layout(int row_tasks, int col_tasks) {
  NoAllocLayout l;
  l.desc = kNoAllocWorkBytes;
  l.state = align256(l.desc + sizeof(MapDesc));
  l.part = align256(l.state + sizeof(MapState));
  l.info = align256(l.part + 2 * sizeof(double) * row_tasks);   // part, part2
  l.ctrl = align256(l.info + sizeof(vs_solve_info));
  l.row_map = align256(l.ctrl + sizeof(Ctrl));
  l.col_map = align256(l.row_map + sizeof(int) * row_tasks);
  l.end = align256(l.col_map + sizeof(int) * col_tasks);
  return l;
}

// Writes the descriptor and zeroes every slot that must start at zero.
__global__ void k_noalloc_init(MapDesc desc, unsigned char* base, NoAllocLayout l) {
  if (blockIdx.x == 0 && threadIdx.x == 0) *reinterpret_cast<MapDesc*>(base + l.desc) = desc;
  for (size_t i = l.state + threadIdx.x; i < l.end; i += blockDim.x) base[i] = 0;
}

std::mutex g_noalloc_mutex;
void* g_noalloc_ptr[64] = {};

}  // namespace

extern "C" int vs_solve_steady_noalloc(vs_kernel k, const float* p_dyn, const float* p_leak0,
                                       const float* s_kappa, const vs_solve_params* params,
                                       float* theta, vs_solve_info* info_host, void* stream) {
  if (!k) return vs_set_error(VS_ERR_INVALID_ARG, "NULL kernel");
  int rc = vs_validate_params(params);
  if (rc) return rc;
  if (vs_params_physics(params))
    return vs_set_error(VS_ERR_INVALID_ARG, "vs_solve_steady_noalloc runs the linear models only");
  if (params->precision != VS_PREC_FP32 || params->engine == VS_ENGINE_CLUSTER)
    return vs_set_error(VS_ERR_INVALID_ARG,
                        "vs_solve_steady_noalloc runs the FP32 streamed engine only (precision "
                        "VS_PREC_FP32, engine VS_ENGINE_AUTO or VS_ENGINE_STREAMED)");
  if (!p_dyn || !p_leak0 || !theta) return vs_set_error(VS_ERR_INVALID_ARG, "NULL map");
  uintptr_t al = (uintptr_t)p_dyn | (uintptr_t)p_leak0 | (uintptr_t)theta | (uintptr_t)s_kappa;
  if (al & 15u) return vs_set_error(VS_ERR_INVALID_ARG, "maps must be 16-byte aligned");
  const int n = k->n;
  if (n > kNoAllocMaxN)
    return vs_set_error(VS_ERR_INVALID_ARG,
                        "vs_solve_steady_noalloc supports n <= %d (got %d): its scratch is a "
                        "fixed %zu-byte device array; use vs_solve_steady for larger grids",
                        kNoAllocMaxN, n, kNoAllocBytes);
  cudaStream_t s = (cudaStream_t)stream;

  // one-time set-up per device: resolve the array's device address
  int dev = 0;
  VS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return vs_set_error(VS_ERR_INVALID_ARG, "device index %d", dev);
  unsigned char* base = nullptr;
  {
    std::lock_guard<std::mutex> lk(g_noalloc_mutex);
    if (!g_noalloc_ptr[dev]) {
      void* ptr = nullptr;
      cudaError_t e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess || !ptr)
        return vs_set_error(VS_ERR_CUDA, "cudaGetSymbolAddress(scratch): %s", cudaGetErrorString(e));
      g_noalloc_ptr[dev] = ptr;
    }
    base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  }

  MapDesc m = {};
  m.p_dyn = p_dyn;
  m.p_leak0 = p_leak0;
  m.s = s_kappa;
  m.theta = theta;
  m.work = reinterpret_cast<float*>(base);
  m.Kt = k->Kt32;
  m.tw4n = k->fft->tw4n;
  m.digrev = k->fft->digrev;
  m.kmax = k->kmax;
  m.n = n;
  m.rb = rows_for(n, 8192);
  m.cb = cols_for(n, 8192);
  const int row_tasks = n / m.rb, col_tasks = n / m.cb;
  NoAllocLayout l = noalloc_layout(row_tasks, col_tasks);
  if (l.end > kNoAllocBytes) return vs_set_error(VS_ERR_INVALID_ARG, "scratch layout overflow");

  const size_t smem = (size_t)(std::max(m.rb, m.cb) / 2) * padded_len(n) * sizeof(float2);
  {
    std::lock_guard<std::mutex> lk(g_attr_mutex);
    if (smem > g_smem_attr_steady) {
      VS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_solve_steady<false>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      VS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_solve_steady<false>,
                                       cudaFuncAttributePreferredSharedMemoryCarveout, 100));
      g_smem_attr_steady = smem;
    }
  }
  int per_sm = 0, sms = 0;
  VS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_solve_steady<false>, kThreads,
                                                            smem));
  VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  if (per_sm < 1) return vs_set_error(VS_ERR_INVALID_ARG, "no block fits on an SM");

  // row/col task -> map index tables are all zero (one map): cleared by init
  k_noalloc_init<<<1, 256, 0, s>>>(m, base, l);
  VS_CUDA_TRY(cudaGetLastError());

  PlanDev P = {};
  P.maps = reinterpret_cast<const MapDesc*>(base + l.desc);
  P.row_map = reinterpret_cast<const int*>(base + l.row_map);
  P.col_map = reinterpret_cast<const int*>(base + l.col_map);
  P.st = reinterpret_cast<MapState*>(base + l.state);
  P.part = reinterpret_cast<double*>(base + l.part);
  P.part2 = P.part + row_tasks;
  P.info = reinterpret_cast<vs_solve_info*>(base + l.info);
  P.ctrl = reinterpret_cast<Ctrl*>(base + l.ctrl);
  P.n_maps = 1;
  P.row_tasks = row_tasks;
  P.col_tasks = col_tasks;
  P.max_iter = params->max_iter;
  P.beta = (float)params->beta_per_K;
  P.alpha = (float)params->alpha_per_K;
  P.tol = (float)params->tol_K;
  P.stop_rule = params->stop_rule;
  P.n_steps = 0;
  P.warm = 0;
  P.adaptive = 1;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(std::max(1, std::min(per_sm * sms, std::max(row_tasks, col_tasks))));
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_solve_steady<false>, P);
  if (e != cudaSuccess)
    return vs_set_error(VS_ERR_CUDA, "cooperative launch: %s", cudaGetErrorString(e));

  vs_solve_info inf;
  unsigned abort_flag = 0;
  VS_CUDA_TRY(cudaMemcpyAsync(&inf, base + l.info, sizeof(inf), cudaMemcpyDeviceToHost, s));
  VS_CUDA_TRY(cudaMemcpyAsync(&abort_flag, base + l.ctrl + offsetof(Ctrl, abort), sizeof(unsigned),
                              cudaMemcpyDeviceToHost, s));
  VS_CUDA_TRY(cudaStreamSynchronize(s));
  if (abort_flag) return vs_set_error(VS_ERR_TIMEOUT, "grid barrier timed out");
  if (info_host) *info_host = inf;
  return inf.status;
}

extern "C" int vs_tc_transform(const float* in, float* out, int rows, int n, int inverse,
                               void* stream) {
  if (!in || !out) return vs_set_error(VS_ERR_INVALID_ARG, "NULL array");
  if (!tc_size_ok(n) || (n & (n - 1)))
    return vs_set_error(VS_ERR_INVALID_ARG, "n must be a power of two in [128, 1024] (got %d)", n);
  if (rows <= 0 || rows % 128) return vs_set_error(VS_ERR_INVALID_ARG, "rows must be a positive multiple of 128");
  if (((uintptr_t)in | (uintptr_t)out) & 15u) return vs_set_error(VS_ERR_INVALID_ARG, "arrays must be 16-byte aligned");
  int st = VS_OK;
  const TcMats* tm = get_tc_mats(n, &st);
  if (!tm) return st;
  VS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_tc_transform,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kTcSmemBytes));
  VS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_tc_transform,
                                   cudaFuncAttributePreferredSharedMemoryCarveout, 100));
  int dev = 0, sms = 0;
  VS_CUDA_TRY(cudaGetDevice(&dev));
  VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  int grid = std::max(1, std::min(sms, rows / 128));
  k_tc_transform<<<grid, kTcThreads, kTcSmemBytes, (cudaStream_t)stream>>>(
      in, out, rows, n, inverse ? tm->inv : tm->fwd);
  VS_CUDA_TRY(cudaGetLastError());
  return VS_OK;
}
