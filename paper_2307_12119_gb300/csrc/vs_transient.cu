// Transient of one map (Sec. IV-D/E: single-pole response per cosine mode,
// Eq. 35, untruncated superposition of power differences, Eq. 36, run as the
// per-mode recursion) with lagged leakage, for grids of 256^2 .. 1024^2.
//
// One persistent cooperative launch of N / R CTAs for the whole trace. CTA c
// owns the rows y in [cR, cR + R) and the x-frequencies p in [cR, cR + R) for
// every step, so everything that belongs to one CTA stays on chip across
// steps:
//   - the recursion state W and the per-mode constants (K - A) / N^2, A / N^2
//     and rho = exp(-dt / tau) of its R x N modes, in shared memory;
//   - P_leak0 of its R rows, in registers (the thread <-> cell mapping of the
//     update is the same every step); s of its rows in shared memory (with
//     implicit leakage or a window that space holds other per-mode state, and
//     s is re-read through the L1 each step).
// Per step, two phases, each ending in an exchange through the spectral map in
// global memory (x-frequency major):
//   column phase: forward DCT along y of its columns, W <- rho W + (1 - rho) X,
//     Y = (K - A) X + A W (the step response (K - A) + A (1 - rho^j) of the
//     primary alias, the finer aliases settled within a step), inverse DCT
//     along y;
//   row phase: inverse DCT along x of its rows -> u_n, theta_n = s u_n /
//     (1 - alpha s u_n) written to the output trace, the next source
//     P_{n+1} = P_dyn,n+1 + P_leak0 (1 + beta theta_n) (its P_dyn loads issued
//     before the inverse transform), forward DCT along x.
// With lagged leakage the exchange needs no grid barrier: every word of the
// map carries, in its upper half, the number of the phase that wrote it, and
// a consumer polls its own words until they carry the phase it waits for (one
// L2 round trip when the data is there, instead of a barrier's arrive, poll
// and then load). One buffer suffices: a CTA overwrites a word only after it
// has received data computed from every read of that word's previous value.
// With implicit leakage every iterate ends in a grid barrier, which also
// carries the iterate's decision. Both waits are bounded spins: on timeout
// the launch sets an abort word and every CTA returns (VS_ERR_TIMEOUT), no
// trap.
#include <math.h>

#include <algorithm>

#include "vs_fft.cuh"
#include "vs_internal.cuh"
#include "vs_solve_common.cuh"

using namespace vsfft;
using vsk::kFlagNonfinite;
using vsk::kFlagRunaway;

namespace {

constexpr int ilog2(int v) { return v <= 1 ? 0 : 1 + ilog2(v / 2); }

constexpr long long kTrSpinLimit = 20000000LL;   // ~ seconds of polling
constexpr long long kTrPollLimit = 4000000LL;    // tag polls (each an L2 round trip): ~ seconds

struct TrCtrl {
  // arrivals so far of the even and of the odd CTAs, each on its own 128-byte
  // line: barrier b is complete when both reach (b + 1) * grid / 2
  unsigned count[2][32];
  unsigned abort;
  int flags;
  // implicit leakage: the iterates' largest change (float bits, two words
  // used alternately), iterations over all steps, the largest final change,
  // and whether a step ended unconverged
  unsigned resid[2];
  int iters;
  float max_resid;
  int growth;
};

struct TrArgs {
  const float* p_dyn;      // [n_steps][N][N]
  const float* p_leak0;    // [N][N]
  const float* s;          // [N][N] or NULL (= 1)
  float* theta;            // [n_steps][N][N]
  float* work;             // [N][N] spectral map, x-frequency major (implicit leakage)
  unsigned long long* xw;  // [N][N] the same map as tagged words (lagged leakage; zeroed)
  const float* Kt;         // [p][q] cosine-basis kernel
  const float* trA;        // [p][q] primary-alias weight
  const float* trRho;      // [p][q] exp(-dt / (C g))
  const float2* tw4n;
  TrCtrl* ctrl;
  int n_steps;
  float beta, alpha;
  float tol;               // implicit leakage: per-step fixed point
  int max_iter;
  int stop_rule;           // VS_STOP_* of that fixed point
  int window;              // WIN: step responses settled from age `window` on (>= 1)
  float* ring;             // WIN, window >= 2: [window - 1][N][N] X - W of the last steps per mode
};

__device__ __forceinline__ unsigned tr_ld_acquire(const unsigned* p) {
  unsigned v;
  asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
  return v;
}

// Grid barrier on two monotonic arrival counters (no reset, so no CTA does
// extra atomics): the even CTAs count on one, the odd ones on the other, and
// barrier b of the launch is complete when each reaches (b + 1) * grid / 2;
// `target` is that value, kept by every CTA. Thread 0 arrives with a release
// add after the block barrier (ordering the block's writes before it), threads
// 0 and 1 wait on one counter each with acquire loads (and record in
// abort_sm[2] whether they gave up); the block barrier after them orders the
// block's next reads. Two counters on separate lines measured
// 1.5 us per barrier on 128 CTAs against 2.3 us for one counter with full
// fences. False if the launch aborted (a bounded wait gave up somewhere).
__device__ bool tr_barrier(TrCtrl* c, unsigned& target, unsigned* abort_sm) {
  __syncthreads();
  target += gridDim.x / 2;
  const int t = threadIdx.x;
  if (t == 0)
    asm volatile("red.release.gpu.global.add.u32 [%0], 1;" ::"l"(&c->count[blockIdx.x & 1][0])
                 : "memory");
  if (t < 2) {
    long long spins = 0;
    unsigned ab = 0u;
    while (tr_ld_acquire(&c->count[t][0]) < target) {
      if ((++spins & 15) == 0 && (ab = tr_ld_acquire(&c->abort)) != 0u) break;
      if (spins > 64) __nanosleep(32);
      if (spins > kTrSpinLimit) {
        atomicExch(&c->abort, 1u);
        ab = 1u;
        break;
      }
    }
    abort_sm[t] = ab;
  }
  __syncthreads();
  return (abort_sm[0] | abort_sm[1]) == 0u;
}

// Tagged words of the lagged exchange: the value's bits in the lower half,
// the number of the phase that wrote it in the upper half. Relaxed accesses at
// GPU scope (served by the L2, never a stale L1 line); an aligned 64-bit access
// is single-copy atomic, and a vector of them is a set of such accesses, so a
// reader sees a value together with its own tag.
__device__ __forceinline__ unsigned long long tr_tag(float v, unsigned tag) {
  return ((unsigned long long)tag << 32) | __float_as_uint(v);
}
__device__ __forceinline__ unsigned tr_tag_of(unsigned long long w) { return (unsigned)(w >> 32); }
__device__ __forceinline__ float tr_val(unsigned long long w) { return __uint_as_float((unsigned)w); }
__device__ __forceinline__ unsigned long long tr_ld64(const unsigned long long* p) {
  unsigned long long v;
  asm volatile("ld.relaxed.gpu.global.b64 %0, [%1];" : "=l"(v) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ ulonglong2 tr_ld128(const unsigned long long* p) {
  ulonglong2 v;
  asm volatile("ld.relaxed.gpu.global.v2.b64 {%0, %1}, [%2];" : "=l"(v.x), "=l"(v.y) : "l"(p) : "memory");
  return v;
}
__device__ __forceinline__ void tr_st64(unsigned long long* p, unsigned long long v) {
  asm volatile("st.relaxed.gpu.global.b64 [%0], %1;" ::"l"(p), "l"(v) : "memory");
}
__device__ __forceinline__ void tr_st128(unsigned long long* p, unsigned long long v0, unsigned long long v1) {
  asm volatile("st.relaxed.gpu.global.v2.b64 [%0], {%1, %2};" ::"l"(p), "l"(v0), "l"(v1) : "memory");
}

// One more round of a bounded tag poll: false once the launch aborted or this
// thread gave up (it then sets the abort word).
__device__ __forceinline__ bool tr_poll_round(TrCtrl* c, long long& spins) {
  ++spins;
  if ((spins & 15) == 0 && tr_ld_acquire(&c->abort) != 0u) return false;
  if (spins > kTrPollLimit) {
    atomicExch(&c->abort, 1u);
    return false;
  }
  if (spins > 2) __nanosleep(64);
  return true;
}

template <int N>
struct TrSched {
  __host__ __device__ static constexpr int radix(int p) {
    if (N == 1024) return p < 2 ? 8 : 16;
    int n = N;
    for (int i = 0; i < p; ++i) n /= (n >= 16 ? 16 : n);
    return n >= 16 ? 16 : n;
  }
  __host__ __device__ static constexpr int passes() {
    int n = N, q = 0;
    while (n > 1) { n /= radix(q); ++q; }
    return q;
  }
  __host__ __device__ static constexpr int len(int p) {
    int L = N;
    for (int i = 0; i < p; ++i) L /= radix(i);
    return L;
  }
  __host__ __device__ static constexpr int tw_off(int p) {
    int o = 0;
    for (int i = 0; i < p; ++i) o += (radix(i) - 1) * (len(i) / radix(i));
    return o;
  }
  static constexpr int TW = tw_off(passes());            // entries of the table (< N)
  // position of frequency k in the forward output (decimation in frequency):
  // its mixed-radix digits, pass 0's least significant, each times the
  // sub-stride L / R of its pass
  __host__ __device__ static constexpr int digit_reversed(int k) {
    int pos = 0;
    for (int p = 0; p < passes(); ++p) {
      pos += (k % radix(p)) * (len(p) / radix(p));
      k /= radix(p);
    }
    return pos;
  }
};

// N x N map, R rows (and R x-frequencies) per CTA, T threads per CTA; a CTA
// of 256 threads is launched two to an SM.
template <int N, int R, int NT>
struct TrShape {
  static constexpr int F = R / 2;                       // complex FFTs per CTA and phase
  static constexpr int THREADS = NT;
  static constexpr int PER_SM = 512 / NT;
  static constexpr int NP = N + N / 16 + 1;
  // row stride of the per-mode arrays: 2 F MS = 32 (mod 32) words, so the
  // F x 32/F (column pair, frequency) items of a warp fall in distinct banks
  static constexpr int MS = N + 16 / F;
  static constexpr int CELLS = F * N / THREADS;          // update items (2 cells) per thread
  // FFT buffers, per-mode arrays, DCT twiddles W_4N^k (k < N), FFT pass
  // twiddles and digit reversal
  static constexpr size_t SMEM = (size_t)F * NP * sizeof(float2) + 4 * (size_t)R * MS * sizeof(float) +
                                 (size_t)N * sizeof(float2) + (size_t)TrSched<N>::TW * sizeof(float2) +
                                 (size_t)N * sizeof(int);
  static_assert(F >= 1 && (F * N) % THREADS == 0 && 16 % F == 0 && THREADS <= F * N &&
                    SMEM * PER_SM <= 225 * 1024, "shape");
};

// One radix-R pass (block length L) over the F in-place FFTs of length N in
// buf (padded stride NP), twiddles from the pass's own table twp. Forward:
// decimation in frequency (butterfly, then W_L^{j r}); inverse: conjugate
// twiddle, then the inverse butterfly.
template <int N, int L, int R, bool FWD>
__device__ __forceinline__ void tr_pass(float2* buf, int nfft, int stride, const float2* twp) {
  constexpr int m = L / R, per = N / R;
  const int total = nfft * per;
  for (int b = threadIdx.x; b < total; b += blockDim.x) {
    const int f = b / per, rem = b % per, blk = rem / m, j = rem % m;
    float2* base = buf + f * stride;
    const int i0 = blk * L + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[pad(i0 + r * m)];
    if (FWD) {
      dftR<R, true>(v);
      if (m > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], twp[(r - 1) * m + j]);
      }
    } else {
      if (m > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmulc(v[r], twp[(r - 1) * m + j]);
      }
      dftR<R, false>(v);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) base[pad(i0 + r * m)] = v[r];
  }
}

template <int N, int P, bool FWD>
__device__ __forceinline__ void tr_pass_p(float2* buf, int nfft, int stride, const float2* ptw) {
  using Q = TrSched<N>;
  tr_pass<N, Q::len(P), Q::radix(P), FWD>(buf, nfft, stride, ptw + Q::tw_off(P));
}

// Forward FFT (natural -> digit-reversed order), a block barrier after each
// pass; FIRST = 1 starts after pass 0 (run by the caller in registers).
template <int N, int FIRST = 0>
__device__ __forceinline__ void tr_fft_forward(float2* buf, int nfft, int stride, const float2* ptw) {
  constexpr int P = TrSched<N>::passes();
  static_assert(P >= 2 && P <= 3, "schedule");
  if constexpr (FIRST == 0) {
    tr_pass_p<N, 0, true>(buf, nfft, stride, ptw);
    __syncthreads();
  }
  tr_pass_p<N, 1, true>(buf, nfft, stride, ptw);
  __syncthreads();
  if constexpr (P == 3) {
    tr_pass_p<N, 2, true>(buf, nfft, stride, ptw);
    __syncthreads();
  }
}

// Inverse FFT (digit-reversed -> natural, unnormalised), passes undone in
// reverse; LAST = 1 stops before pass 0 (left to the caller).
template <int N, int LAST = 0>
__device__ __forceinline__ void tr_fft_inverse(float2* buf, int nfft, int stride, const float2* ptw) {
  constexpr int P = TrSched<N>::passes();
  if constexpr (P == 3) {
    tr_pass_p<N, 2, false>(buf, nfft, stride, ptw);
    __syncthreads();
  }
  tr_pass_p<N, 1, false>(buf, nfft, stride, ptw);
  __syncthreads();
  if constexpr (LAST == 0) {
    tr_pass_p<N, 0, false>(buf, nfft, stride, ptw);
    __syncthreads();
  }
}

// IMPL: implicit leakage (the leakage of step n at theta_n): each step
// iterates the column and row phases from theta_{n-1} until the stopping rule
// holds on the largest change (<= tol, or its error estimate from the step's
// last two changes) or max_iter, the recursion state W committed with the
// source of the step's last iterate; the decision of an iterate is read by
// every CTA from the same word after a grid barrier.
// WIN: the window of Sec. IV-E with lagged leakage: step responses older than
// `window` steps are taken as settled, S_j = K for j >= window, so a mode's
// response is Y_n = K X_n - A sum_{0 < j < window} rho^j (X_{n-j+1} - X_{n-j}),
// computed from the untruncated recursion and a ring of its last window - 1
// differences X_m - W_m per mode (slot m mod (window - 1), in global memory:
// the CTA's own modes, L2-resident); window 1 is the settled response K X_n.
template <int N, int R, int NT, bool IMPL, bool WIN = false>
__global__ void __launch_bounds__(NT, 512 / NT) k_transient_fast(TrArgs a) {
  using S = TrShape<N, R, NT>;
  constexpr int F = S::F, NP = S::NP, MS = S::MS, T = S::THREADS, CELLS = S::CELLS, half = N / 2;
  constexpr int lgN = ilog2(N), lgF = ilog2(F);
  constexpr bool TAG = !IMPL;   // exchange by tagged words instead of grid barriers
  static_assert(!(IMPL && WIN) && (!WIN || (R * N) % T == 0), "variant");
  extern __shared__ __align__(16) float2 tr_smem[];
  __shared__ int red_i[T / 32];
  __shared__ unsigned abort_sm[2];
  __shared__ int tag_abort;
  float2* buf = tr_smem;                                  // [F][NP]
  float* km = reinterpret_cast<float*>(buf + F * NP);     // [R][MS] (K - A) / N^2
  float* am = km + R * MS;                                // [R][MS] A / N^2
  float* rh = am + R * MS;                                // [R][MS] rho
  float* W = rh + R * MS;                                 // [R][MS] recursion state
  float2* tw = reinterpret_cast<float2*>(W + R * MS);     // [N] DCT twiddles W_4N^k
  float2* ptw = tw + N;                                   // [TW] FFT pass twiddles
  int* dr = reinterpret_cast<int*>(ptw + TrSched<N>::TW); // [N] digit reversal
  float* Xs = reinterpret_cast<float*>(dr + N);           // [R][MS] IMPL: the last source;
                                                          // WIN: X - W of `window - 1` steps ago;
                                                          // otherwise s of the CTA's rows
  constexpr bool S_SMEM = !IMPL && !WIN;                  // s read from shared memory
  // s of rows y0 + 2f (.x) and y0 + 2f + 1 (.y) at x, for the update
  const float2* s2 = reinterpret_cast<const float2*>(Xs);
  const int tid = threadIdx.x;
  const int y0 = blockIdx.x * R, p0 = blockIdx.x * R;
  const size_t nn = (size_t)N * N;
  if (tid == 0) tag_abort = 0;
  for (int i = tid; i < N; i += T) {
    tw[i] = __ldg(&a.tw4n[i]);
    dr[i] = TrSched<N>::digit_reversed(i);
  }
  {
    // W_L^{j r} = W_4N^{j r 4N / L}, pass by pass
    using Q = TrSched<N>;
#pragma unroll
    for (int p = 0; p < Q::passes(); ++p) {
      const int L = Q::len(p), Rp = Q::radix(p), m = L / Rp, o = Q::tw_off(p);
      if (m == 1) continue;
      for (int e = tid; e < (Rp - 1) * m; e += T) {
        const int r = e / m + 1, j = e % m;
        ptw[o + e] = __ldg(&a.tw4n[j * r * (4 * N / L)]);
      }
    }
  }
  const float inv_n2 = 1.f / ((float)N * (float)N);
  const float beta = a.beta, alpha = a.alpha;

  for (int i = tid; i < R * N; i += T) {
    const int c = i >> lgN, q = i & (N - 1), o = c * MS + q;
    const size_t g = (size_t)(p0 + c) * N + q;
    const float A = __ldg(&a.trA[g]), K = __ldg(&a.Kt[g]);
    km[o] = (K - A) * inv_n2;
    am[o] = A * inv_n2;
    rh[o] = __ldg(&a.trRho[g]);
    W[o] = 0.f;
  }
  // This thread's cells: item j -> (f, x), rows y0 + 2f (.x) and y0 + 2f + 1
  // (.y). FUSE (lagged leakage, pass 0 of the schedule one butterfly per
  // thread): the cells of this thread's pass-0 butterfly, the Makhoul
  // positions jj + j M0 of FFT f, so that the row phase runs the inverse
  // pass 0, the update and the forward pass 0 in registers; otherwise
  // consecutive cells of a row.
  constexpr int R0 = TrSched<N>::radix(0), M0 = N / R0;
  constexpr bool FUSE = !IMPL && F * M0 == T && R0 == CELLS;
  auto cell = [&](int j, int& f, int& x) {
    if constexpr (FUSE) {
      f = tid / M0;
      const int p = tid % M0 + j * M0;
      x = p < half ? 2 * p : 2 * (N - 1 - p) + 1;
    } else {
      const int it = tid + j * T;
      f = it >> lgN;
      x = it & (N - 1);
    }
  };
  if constexpr (S_SMEM) {
    // s is the same every step: its cells stay in shared memory, item j of
    // thread t at j T + t
    if (a.s) {
      float2* sw = reinterpret_cast<float2*>(Xs);
#pragma unroll
      for (int j = 0; j < CELLS; ++j) {
        int f, x;
        cell(j, f, x);
        const size_t g = (size_t)(y0 + 2 * f) * N + x;
        sw[j * T + tid] = make_float2(__ldg(&a.s[g]), __ldg(&a.s[g + N]));
      }
    }
  }
  float2 pl[CELLS], pd[CELLS];
#pragma unroll
  for (int j = 0; j < CELLS; ++j) {
    int f, x;
    cell(j, f, x);
    const size_t i0 = (size_t)(y0 + 2 * f) * N + x, i1 = i0 + N;
    pl[j] = make_float2(__ldg(&a.p_leak0[i0]), __ldg(&a.p_leak0[i1]));
    pd[j] = make_float2(__ldg(&a.p_dyn[i0]), __ldg(&a.p_dyn[i1]));
  }
  int flags = 0;
  unsigned target = 0;    // arrivals that complete the next grid barrier
  unsigned ex = 0;        // TAG: phases completed so far (the tag of the data last written)

  // forward DCT along x of the source in buf (Makhoul order), stored
  // x-frequency major; from1: pass 0 is done (FUSE)
  auto row_forward = [&](bool from1) {
    __syncthreads();
    if (from1)
      tr_fft_forward<N, 1>(buf, F, NP, ptw);
    else
      tr_fft_forward<N, 0>(buf, F, NP, ptw);
    for (int it = tid; it < F * (half + 1); it += T) {
      const int f = it & (F - 1), k = it >> lgF, nk = N - k;
      const float2 zk = buf[f * NP + pad(dr[k])];
      const float2 znk = buf[f * NP + pad(dr[k == 0 ? 0 : nk])];
      const float2 vk = dct_post(zk, znk, tw[k]);
      if constexpr (TAG) {
        tr_st128(a.xw + (size_t)k * N + y0 + 2 * f, tr_tag(vk.x, ex + 1), tr_tag(vk.y, ex + 1));
      } else {
        *reinterpret_cast<float2*>(a.work + (size_t)k * N + y0 + 2 * f) = vk;
      }
      if (k != 0 && k != half) {
        const float2 vn = dct_post(znk, zk, tw[nk]);
        if constexpr (TAG) {
          tr_st128(a.xw + (size_t)nk * N + y0 + 2 * f, tr_tag(vn.x, ex + 1), tr_tag(vn.y, ex + 1));
        } else {
          *reinterpret_cast<float2*>(a.work + (size_t)nk * N + y0 + 2 * f) = vn;
        }
      }
    }
  };
  // the end of a phase: TAG, the next phase's data carries tag ex + 1;
  // otherwise a grid barrier. False if the launch aborted.
  auto exchange = [&]() -> bool {
    if constexpr (TAG) {
      ++ex;
      return true;
    } else {
      return tr_barrier(a.ctrl, target, abort_sm);
    }
  };

  // step 0: the first source P_1 = P_dyn,1 + P_leak0 (theta_0 = 0)
#pragma unroll
  for (int j = 0; j < CELLS; ++j) {
    int f, x;
    cell(j, f, x);
    buf[f * NP + pad(makhoul_pos(x, N))] = make_float2(pd[j].x + pl[j].x, pd[j].y + pl[j].y);
  }
  row_forward(false);
  if (!exchange()) return;

  // IMPL: the iterate of the current step, whether the previous step is still
  // to be committed into W, the previous iterate of this thread's cells
  // (theta_{n-1} at the first iterate) and the iterate count of the launch
  int iter = 1, g = 0;
  bool commit = false;
  float prev_r = INFINITY;   // IMPL: the previous change of the current step
  float2 thp[IMPL ? CELLS : 1];
#pragma unroll
  for (int j = 0; j < (IMPL ? CELLS : 1); ++j) thp[j] = make_float2(0.f, 0.f);
  __shared__ float dec_r;
  __shared__ int dec_f;

  for (int step = 1; step <= a.n_steps;) {
    // ---- column phase: this CTA's x-frequency columns p0 .. p0 + R - 1
    {
      float2 c[CELLS];   // all loads of a thread issued before the stores
      // WIN: X - W of this CTA's modes from `window - 1` steps ago (rows p0 ..
      // of the ring slot this step overwrites), loaded while the phase polls
      constexpr int RG = WIN ? R * N / T : 1;
      float rg[RG];
      if constexpr (WIN) {
        if (a.window >= 2) {
          const float* src = a.ring + (size_t)(step % (a.window - 1)) * nn + (size_t)p0 * N;
#pragma unroll
          for (int u = 0; u < RG; ++u) rg[u] = __ldcg(src + tid + u * T);
        }
      }
      if constexpr (TAG) {
        // poll this thread's words until they carry phase ex, then (block
        // barrier: the previous phase's reads of buf are done) stage them
        unsigned long long wa[CELLS], wb[CELLS];
        auto col = [&](int q, int h) {
          const int it = tid + q * T, f = it >> lgN, j = it & (N - 1);
          return a.xw + (size_t)(p0 + 2 * f + h) * N + j;
        };
#pragma unroll
        for (int q = 0; q < CELLS; ++q) {
          wa[q] = tr_ld64(col(q, 0));
          wb[q] = tr_ld64(col(q, 1));
        }
        long long spins = 0;
        for (;;) {
          bool ready = true;
#pragma unroll
          for (int q = 0; q < CELLS; ++q) ready &= tr_tag_of(wa[q]) == ex && tr_tag_of(wb[q]) == ex;
          if (ready) break;
          if (!tr_poll_round(a.ctrl, spins)) {
            tag_abort = 1;
            break;
          }
#pragma unroll
          for (int q = 0; q < CELLS; ++q) {
            if (tr_tag_of(wa[q]) != ex) wa[q] = tr_ld64(col(q, 0));
            if (tr_tag_of(wb[q]) != ex) wb[q] = tr_ld64(col(q, 1));
          }
        }
#pragma unroll
        for (int q = 0; q < CELLS; ++q) c[q] = make_float2(tr_val(wa[q]), tr_val(wb[q]));
        __syncthreads();
        if (tag_abort) return;
        if constexpr (WIN) {
          if (a.window >= 2) {
#pragma unroll
            for (int u = 0; u < RG; ++u) {
              const int i = tid + u * T;
              Xs[(i >> lgN) * MS + (i & (N - 1))] = rg[u];
            }
          }
        }
      } else {
#pragma unroll
        for (int q = 0; q < CELLS; ++q) {
          const int it = tid + q * T, f = it >> lgN, j = it & (N - 1);
          c[q] = make_float2(a.work[(size_t)(p0 + 2 * f) * N + j], a.work[(size_t)(p0 + 2 * f + 1) * N + j]);
        }
      }
#pragma unroll
      for (int q = 0; q < CELLS; ++q) {
        const int it = tid + q * T, f = it >> lgN, j = it & (N - 1);
        buf[f * NP + pad(makhoul_pos(j, N))] = c[q];
      }
    }
    __syncthreads();
    tr_fft_forward<N>(buf, F, NP, ptw);
    for (int it = tid; it < F * (half + 1); it += T) {
      // a warp takes F column pairs x 32/F consecutive frequencies: the FFT
      // outputs (blocks of odd padded stride) and the mode arrays (row stride
      // MS) are then both read without bank conflicts
      const int f = it & (F - 1), k = it >> lgF, nk = N - k;
      const int ia = f * NP + pad(dr[k]);
      const int ib = f * NP + pad(dr[k == 0 ? 0 : nk]);
      const float2 zk = buf[ia], znk = buf[ib];
      const float2 xk = dct_post(zk, znk, tw[k]);
      auto mode = [&](int c, int q, float x) {
        const int i = c * MS + q;
        if constexpr (WIN) {
          const float Ks = km[i] + am[i];         // K / N^2
          const int Rw = a.window - 1;
          if (Rw == 0) return Ks * x;
          // the truncated sum as the untruncated one minus its value Rw steps
          // back: with S_m = X_m - W_m (W the recursion of the untruncated
          // response), sum_{j=1..Rw} rho^j (X_{n-j+1} - X_{n-j}) =
          // S_n - rho^Rw S_{n-Rw}; the ring holds S of the last Rw steps per
          // mode (zero before the first step), S_{n-Rw} in the slot S_n takes
          // (loaded into Xs at the start of the phase, so that no load of a
          // ring word is pending when it is overwritten)
          const float rho = rh[i];
          const float w = fmaf(rho, W[i] - x, x);
          W[i] = w;
          float rp = rho;
          for (int j = 1; j < Rw; ++j) rp *= rho;
          const float s_now = x - w;
          const float acc = fmaf(-rp, Xs[i], s_now);
          __stcg(a.ring + (size_t)(step % Rw) * nn + (size_t)(p0 + c) * N + q, s_now);
          return fmaf(Ks, x, -am[i] * acc);
        } else if constexpr (IMPL) {
          // W stays at the last committed step; the step before this one is
          // committed (with its last source) at its first column phase
          float Wc = W[i];
          if (commit) {
            Wc = fmaf(rh[i], Wc - Xs[i], Xs[i]);
            W[i] = Wc;
          }
          Xs[i] = x;
          const float w = fmaf(rh[i], Wc - x, x);
          return fmaf(km[i], x, am[i] * w);
        } else {
          const float w = fmaf(rh[i], W[i] - x, x);
          W[i] = w;
          return fmaf(km[i], x, am[i] * w);
        }
      };
      const float2 yk = make_float2(mode(2 * f, k, xk.x), mode(2 * f + 1, k, xk.y));
      float2 ynk;
      if (k != 0 && k != half) {
        const float2 xnk = dct_post(znk, zk, tw[nk]);
        ynk = make_float2(mode(2 * f, nk, xnk.x), mode(2 * f + 1, nk, xnk.y));
      } else {
        ynk = k == half ? yk : make_float2(0.f, 0.f);
      }
      buf[ia] = dct_pre(yk.x, ynk.x, yk.y, ynk.y, tw[k]);
      if (k != 0 && k != half) buf[ib] = dct_pre(ynk.x, yk.x, ynk.y, yk.y, tw[nk]);
    }
    __syncthreads();
    tr_fft_inverse<N>(buf, F, NP, ptw);
    for (int it = tid; it < F * N; it += T) {
      const int f = it >> lgN, j = it & (N - 1);
      const float2 v = buf[f * NP + pad(makhoul_pos(j, N))];
      if constexpr (TAG) {
        tr_st64(a.xw + (size_t)(p0 + 2 * f) * N + j, tr_tag(v.x, ex + 1));
        tr_st64(a.xw + (size_t)(p0 + 2 * f + 1) * N + j, tr_tag(v.y, ex + 1));
      } else {
        a.work[(size_t)(p0 + 2 * f) * N + j] = v.x;
        a.work[(size_t)(p0 + 2 * f + 1) * N + j] = v.y;
      }
    }
    commit = false;
    if (!exchange()) return;

    // ---- row phase: rows y0 .. y0 + R - 1
    const bool more = step < a.n_steps;
    if (!IMPL && more) {
      // the next power map, loaded while the inverse transform runs
      const float* pdn = a.p_dyn + (size_t)step * nn;
#pragma unroll
      for (int j = 0; j < CELLS; ++j) {
        int f, x;
        cell(j, f, x);
        const size_t i0 = (size_t)(y0 + 2 * f) * N + x;
        pd[j] = make_float2(__ldg(&pdn[i0]), __ldg(&pdn[i0 + N]));
      }
    }
    {
      // the spectra of this CTA's rows at x-frequencies k and N - k, k <= N/2:
      // all loads of a thread issued before the pre-twiddles
      constexpr int PRE = (F * (half + 1) + T - 1) / T;
      float2 xk[PRE], xnk[PRE];
      if constexpr (TAG) {
        // the words of frequencies k and N - k (absent ones pre-tagged as ready)
        ulonglong2 wk[PRE], wn[PRE];
        const unsigned long long zero = tr_tag(0.f, ex);
        auto row = [&](int q, bool other) {
          const int it = tid + q * T, f = it & (F - 1), k = it >> lgF;
          return a.xw + (size_t)(other ? N - k : k) * N + y0 + 2 * f;
        };
        auto has_k = [&](int q) { return tid + q * T < F * (half + 1); };
        auto has_nk = [&](int q) { return has_k(q) && ((tid + q * T) >> lgF) != 0; };
#pragma unroll
        for (int q = 0; q < PRE; ++q) {
          wk[q] = wn[q] = make_ulonglong2(zero, zero);
          if (has_k(q)) wk[q] = tr_ld128(row(q, false));
          if (has_nk(q)) wn[q] = tr_ld128(row(q, true));
        }
        auto ok = [&](const ulonglong2& w) { return tr_tag_of(w.x) == ex && tr_tag_of(w.y) == ex; };
        long long spins = 0;
        for (;;) {
          bool ready = true;
#pragma unroll
          for (int q = 0; q < PRE; ++q) ready &= ok(wk[q]) && ok(wn[q]);
          if (ready) break;
          if (!tr_poll_round(a.ctrl, spins)) {
            tag_abort = 1;
            break;
          }
#pragma unroll
          for (int q = 0; q < PRE; ++q) {
            if (!ok(wk[q])) wk[q] = tr_ld128(row(q, false));
            if (!ok(wn[q])) wn[q] = tr_ld128(row(q, true));
          }
        }
#pragma unroll
        for (int q = 0; q < PRE; ++q) {
          xk[q] = make_float2(tr_val(wk[q].x), tr_val(wk[q].y));
          xnk[q] = make_float2(tr_val(wn[q].x), tr_val(wn[q].y));
        }
        __syncthreads();
        if (tag_abort) return;
      } else {
#pragma unroll
        for (int q = 0; q < PRE; ++q) {
          const int it = tid + q * T, f = it & (F - 1), k = it >> lgF;
          xk[q] = xnk[q] = make_float2(0.f, 0.f);
          if (it < F * (half + 1)) {
            xk[q] = *reinterpret_cast<const float2*>(a.work + (size_t)k * N + y0 + 2 * f);
            if (k != 0) xnk[q] = *reinterpret_cast<const float2*>(a.work + (size_t)(N - k) * N + y0 + 2 * f);
          }
        }
      }
#pragma unroll
      for (int q = 0; q < PRE; ++q) {
        const int it = tid + q * T, f = it & (F - 1), k = it >> lgF, nk = N - k;
        if (it >= F * (half + 1)) continue;
        buf[f * NP + pad(dr[k])] = dct_pre(xk[q].x, xnk[q].x, xk[q].y, xnk[q].y, tw[k]);
        if (k != 0 && k != half)
          buf[f * NP + pad(dr[nk])] = dct_pre(xnk[q].x, xk[q].x, xnk[q].y, xk[q].y, tw[nk]);
      }
    }
    __syncthreads();
    float* th_out = a.theta + (size_t)(step - 1) * nn;
    float resid = 0.f;
    if constexpr (FUSE) {
      tr_fft_inverse<N, 1>(buf, F, NP, ptw);
      // this thread's pass-0 butterfly: inverse, the update of its cells, and
      // (unless this was the last step) the forward butterfly of the next
      // source, in registers and in place
      const int jj = tid % M0;
      float2* base = buf + (tid / M0) * NP;
      float2 v[R0];
#pragma unroll
      for (int r = 0; r < R0; ++r) v[r] = base[pad(jj + r * M0)];
#pragma unroll
      for (int r = 1; r < R0; ++r) v[r] = cmulc(v[r], ptw[(r - 1) * M0 + jj]);
      dftR<R0, false>(v);
#pragma unroll
      for (int j = 0; j < CELLS; ++j) {
        int f, x;
        cell(j, f, x);
        const size_t i0 = (size_t)(y0 + 2 * f) * N + x;
        const float2 u = v[j];
        const float2 sk = !a.s ? make_float2(1.f, 1.f)
                          : S_SMEM ? s2[j * T + tid]
                                   : make_float2(__ldg(&a.s[i0]), __ldg(&a.s[i0 + N]));
        float th[2], q[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
          const float uu = h ? u.y : u.x, S = h ? sk.y : sk.x;
          const float den = fmaf(-alpha * S, uu, 1.f);
          if (!(den > 0.05f)) flags |= kFlagRunaway;
          th[h] = S * uu / den;
          if (!isfinite(th[h])) flags |= kFlagNonfinite;
          const float L0 = h ? pl[j].y : pl[j].x, D = h ? pd[j].y : pd[j].x;
          q[h] = D + L0 * fmaf(beta, th[h], 1.f);
        }
        th_out[i0] = th[0];
        th_out[i0 + N] = th[1];
        v[j] = make_float2(q[0], q[1]);
      }
      if (!more) break;
      dftR<R0, true>(v);
#pragma unroll
      for (int r = 1; r < R0; ++r) v[r] = cmul(v[r], ptw[(r - 1) * M0 + jj]);
#pragma unroll
      for (int r = 0; r < R0; ++r) base[pad(jj + r * M0)] = v[r];
      row_forward(true);
      if (!exchange()) return;
      ++step;
      continue;
    }
    // not FUSE (the other grids, implicit leakage): the whole inverse
    // transform through shared memory, then the update from there
    tr_fft_inverse<N>(buf, F, NP, ptw);
#pragma unroll
    for (int j = 0; j < CELLS; ++j) {
      int f, x;
      cell(j, f, x);
      const int pos = f * NP + pad(makhoul_pos(x, N));
      const size_t i0 = (size_t)(y0 + 2 * f) * N + x;
      const float2 u = buf[pos];
      const float2 sk = !a.s ? make_float2(1.f, 1.f)
                        : S_SMEM ? s2[j * T + tid]
                                 : make_float2(__ldg(&a.s[i0]), __ldg(&a.s[i0 + N]));
      float th[2], q[2];
#pragma unroll
      for (int h = 0; h < 2; ++h) {
        const float uu = h ? u.y : u.x, S = h ? sk.y : sk.x;
        const float den = fmaf(-alpha * S, uu, 1.f);
        if (!(den > 0.05f)) flags |= kFlagRunaway;
        th[h] = S * uu / den;
        if (!isfinite(th[h])) flags |= kFlagNonfinite;
        const float L0 = h ? pl[j].y : pl[j].x, D = h ? pd[j].y : pd[j].x;
        q[h] = D + L0 * fmaf(beta, th[h], 1.f);
      }
      th_out[i0] = th[0];
      th_out[i0 + N] = th[1];
      if constexpr (IMPL) {
        const float2 o = thp[IMPL ? j : 0];
        if (isfinite(th[0])) resid = fmaxf(resid, fabsf(th[0] - o.x));
        if (isfinite(th[1])) resid = fmaxf(resid, fabsf(th[1] - o.y));
        thp[IMPL ? j : 0] = make_float2(th[0], th[1]);
      } else {
        buf[pos] = make_float2(q[0], q[1]);
      }
    }
    if constexpr (!IMPL) {
      if (!more) break;
      row_forward(false);
      if (!exchange()) return;
      ++step;
    } else {
      // the decision of this iterate: its largest change over the map and the
      // flags, gathered on the control words and read back after a barrier
      const int cur = g & 1;
      ++g;
      float rb = resid;
      int fb = flags;
      for (int o = 16; o > 0; o >>= 1) {
        rb = fmaxf(rb, __shfl_down_sync(0xffffffffu, rb, o));
        fb |= __shfl_down_sync(0xffffffffu, fb, o);
      }
      if ((tid & 31) == 0) red_i[tid >> 5] = fb;
      if ((tid & 31) == 0) atomicMax(&a.ctrl->resid[cur], __float_as_uint(rb));
      __syncthreads();
      if (tid == 0) {
        int fo = 0;
        for (int w = 0; w < T / 32; ++w) fo |= red_i[w];
        if (fo) atomicOr(&a.ctrl->flags, fo);
      }
      if (!tr_barrier(a.ctrl, target, abort_sm)) return;
      if (tid == 0) {
        dec_r = __uint_as_float(tr_ld_acquire(&a.ctrl->resid[cur]));
        dec_f = (int)tr_ld_acquire(reinterpret_cast<const unsigned*>(&a.ctrl->flags));
      }
      __syncthreads();
      const float r = dec_r;
      const bool conv = vsk::converged(r, prev_r, iter, a.tol, a.stop_rule);
      const bool done = conv || iter >= a.max_iter || (dec_f & kFlagNonfinite);
      prev_r = done ? INFINITY : r;
      if (blockIdx.x == 0 && tid == 0) {
        // every CTA read the other word one iterate ago, before this iterate's barriers
        a.ctrl->resid[cur ^ 1] = 0u;
        if (done) {
          a.ctrl->iters += iter;
          a.ctrl->max_resid = fmaxf(a.ctrl->max_resid, r);
          if (!conv) a.ctrl->growth = 1;
        }
      }
      if (done && step == a.n_steps) break;
      if (done) {
        // the next step's power, its source at this step's temperature
        const float* pdn = a.p_dyn + (size_t)step * nn;
#pragma unroll
        for (int j = 0; j < CELLS; ++j) {
          int f, x;
          cell(j, f, x);
          const size_t i0 = (size_t)(y0 + 2 * f) * N + x;
          pd[j] = make_float2(__ldg(&pdn[i0]), __ldg(&pdn[i0 + N]));
        }
      }
#pragma unroll
      for (int j = 0; j < CELLS; ++j) {
        int f, x;
        cell(j, f, x);
        const float2 th = thp[IMPL ? j : 0];
        buf[f * NP + pad(makhoul_pos(x, N))] =
            make_float2(pd[j].x + pl[j].x * fmaf(beta, th.x, 1.f), pd[j].y + pl[j].y * fmaf(beta, th.y, 1.f));
      }
      row_forward(false);
      if (!tr_barrier(a.ctrl, target, abort_sm)) return;
      if (done) {
        ++step;
        iter = 1;
        commit = true;
      } else {
        ++iter;
      }
    }
  }
  // flags of the whole launch
  for (int o = 16; o > 0; o >>= 1) flags |= __shfl_down_sync(0xffffffffu, flags, o);
  if ((tid & 31) == 0) red_i[tid >> 5] = flags;
  __syncthreads();
  if (tid == 0) {
    int fo = 0;
    for (int w = 0; w < T / 32; ++w) fo |= red_i[w];
    if (fo) atomicOr(&a.ctrl->flags, fo);
  }
}

template <int N, int R, int NT, bool IMPL, bool WIN = false>
int launch_fast(const TrArgs& args, cudaStream_t s) {
  using S = TrShape<N, R, NT>;
  // one more [R][MS] array: the step's last source (implicit leakage), the
  // window's X - W from `window - 1` steps ago, or s of the CTA's rows
  constexpr size_t smem = S::SMEM + 4 * (size_t)R * S::MS;
  static_assert(smem <= 227 * 1024, "shared memory");
  VS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_transient_fast<N, R, NT, IMPL, WIN>,
                                   cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  int dev = 0, sms = 0, per_sm = 0;
  VS_CUDA_TRY(cudaGetDevice(&dev));
  VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  VS_CUDA_TRY(cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_transient_fast<N, R, NT, IMPL, WIN>,
                                                            S::THREADS, smem));
  const int grid = N / R;
  if (per_sm * sms < grid) return -1;          // not co-resident: the caller falls back
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(grid);
  cfg.blockDim = dim3(S::THREADS);
  cfg.dynamicSmemBytes = smem;
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeCooperative;
  attr[0].val.cooperative = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_transient_fast<N, R, NT, IMPL, WIN>, args);
  if (e != cudaSuccess) return vs_set_error(VS_ERR_CUDA, "transient launch: %s", cudaGetErrorString(e));
  return VS_OK;
}

}  // namespace

bool vs_transient_fast_ok(int n) { return n == 256 || n == 512 || n == 1024; }

// Runs the untruncated transient of one map on the persistent kernel above,
// with lagged leakage or (implicit) the leakage of each step at its own
// temperature. Returns VS_OK and fills *info, a vs_status, or -1 when the
// launch shape does not fit the device (the caller then uses the general
// engine). Allocates its spectral map (tagged words for lagged leakage, zeroed
// so that no word carries a phase number yet) and control words per call.
int vs_transient_fast(vs_kernel k, int n_steps, const float* p_dyn_trace, const float* p_leak0,
                      const float* s_kappa, const vs_solve_params* params, int implicit,
                      int window, float* theta_trace, vs_solve_info* info, cudaStream_t s) {
  const int n = k->n;
  const size_t nn = (size_t)n * n;
  float* work = nullptr;
  TrCtrl* ctrl = nullptr;
  // the spectral map (8 bytes a word), and for a window of 2 or more the ring
  // of past sources
  const size_t ring_maps = window >= 2 ? (size_t)(window - 1) : 0;
  VS_CUDA_TRY(cudaMalloc(&work, sizeof(unsigned long long) * nn + sizeof(float) * nn * ring_maps));
  cudaError_t e = cudaMalloc(&ctrl, sizeof(TrCtrl));
  if (e != cudaSuccess) {
    cudaFree(work);
    return vs_set_error(VS_ERR_OOM, "transient control words: %s", cudaGetErrorString(e));
  }
  TrArgs a = {};
  a.p_dyn = p_dyn_trace;
  a.p_leak0 = p_leak0;
  a.s = s_kappa;
  a.theta = theta_trace;
  a.work = work;
  a.xw = reinterpret_cast<unsigned long long*>(work);
  a.Kt = k->Kt32;
  a.trA = k->trA;
  a.trRho = k->trRho;
  a.tw4n = k->fft->tw4n;
  a.ctrl = ctrl;
  a.n_steps = n_steps;
  a.beta = (float)params->beta_per_K;
  a.alpha = (float)params->alpha_per_K;
  a.tol = (float)params->tol_K;
  a.max_iter = params->max_iter;
  a.stop_rule = params->stop_rule;
  a.window = window;
  a.ring = ring_maps ? work + 2 * nn : nullptr;
  int rc = VS_OK;
  e = cudaMemsetAsync(ctrl, 0, sizeof(TrCtrl), s);
  if (e == cudaSuccess && !implicit) e = cudaMemsetAsync(a.xw, 0, sizeof(unsigned long long) * nn, s);
  if (e == cudaSuccess && ring_maps)
    e = cudaMemsetAsync(a.ring, 0, sizeof(float) * nn * ring_maps, s);
  if (e != cudaSuccess) rc = vs_set_error(VS_ERR_CUDA, "memset: %s", cudaGetErrorString(e));
  if (rc == VS_OK) {
    // lagged (untruncated or windowed) or implicit (untruncated)
    switch (n) {
      case 256:
        rc = implicit ? launch_fast<256, 2, 256, true>(a, s)
             : window ? launch_fast<256, 2, 256, false, true>(a, s) : launch_fast<256, 2, 256, false>(a, s);
        break;
      case 512:
        rc = implicit ? launch_fast<512, 4, 512, true>(a, s)
             : window ? launch_fast<512, 4, 512, false, true>(a, s) : launch_fast<512, 4, 512, false>(a, s);
        break;
      default:
        rc = implicit ? launch_fast<1024, 8, 512, true>(a, s)
             : window ? launch_fast<1024, 8, 512, false, true>(a, s) : launch_fast<1024, 8, 512, false>(a, s);
        break;
    }
  }
  TrCtrl hc = {};
  if (rc == VS_OK) {
    e = cudaMemcpyAsync(&hc, ctrl, sizeof(TrCtrl), cudaMemcpyDeviceToHost, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) rc = vs_set_error(VS_ERR_CUDA, "transient: %s", cudaGetErrorString(e));
  }
  cudaStreamSynchronize(s);
  cudaFree(work);
  cudaFree(ctrl);
  if (rc != VS_OK) return rc;
  if (hc.abort) return vs_set_error(VS_ERR_TIMEOUT, "transient exchange timed out");
  info->status = (hc.flags & kFlagNonfinite) ? VS_ERR_NONFINITE
                 : (hc.flags & kFlagRunaway) ? VS_ERR_RUNAWAY
                 : (implicit && hc.growth) ? VS_ERR_NO_CONVERGENCE : VS_OK;
  info->iterations = implicit ? hc.iters : n_steps;
  info->residual_K = implicit ? (double)hc.max_resid : 0.0;
  info->mu_W = 0.0;
  info->fell_back = 0;
  return info->status;
}
