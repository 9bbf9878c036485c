// Split-precision tensor-core engine that keeps each 256 x 256 map on chip:
// one cluster of two CTAs per map, the steady fixed point (Eqs. 13-21 with the
// convergence loop of Sec. V-C) iterated with every cosine transform (Sec. IV-F
// images) as BF16 hi/lo tcgen05 GEMMs with FP32 accumulation in tensor memory.
//
// Even/odd symmetry. With C[k][j] = cos(pi k (2j + 1) / 2n), C[k][n-1-j] =
// (-1)^k C[k][j], so a length-n DCT-II splits into two half-size products,
//   X[2m]   = sum_{j<h} (x[j] + x[n-1-j]) C[2m][j],
//   X[2m+1] = sum_{j<h} (x[j] - x[n-1-j]) C[2m+1][j]      (h = n/2),
// and its inverse x[j] = sum_k w_k X[k] C[k][j] (w_0 = 1, else 2) into
//   x[j] = E[j] + O[j], x[n-1-j] = E[j] - O[j],
//   E[j] = sum_m w_2m X[2m] C[2m][j], O[j] = sum_m 2 X[2m+1] C[2m+1][j].
// Every transform is two M = 128, N = 128, K = 128 GEMMs, half the work of the
// full N x N product. The constants Cf_e[m][j] = C[2m][j], Cf_o[m][j] =
// C[2m+1][j], Ci_e[j][m] = w_2m C[2m][j], Ci_o[j][m] = 2 C[2m+1][j] are split
// into BF16 hi + lo on the host and streamed from L2 in K-chunks of 16 (1-D
// bulk copies); the product is A_hi B_hi + A_hi B_lo + A_lo B_hi. The 1/n^2 of
// the two inverse transforms sits in the spectral multiplier.
//
// Ownership in the pair (CTA rank c): the row pairs (y', n-1-y') with y' in
// [64c, 64c + 64) (local row r < 64 is y', r + 64 its mirror), and the
// x-frequencies p in [128c, 128c + 128). One iteration, with every operand
// written by an epilogue directly in the K-major layout the next GEMM reads:
//   GEMM 1 (inverse x)      E1/O1[r][j]   = V_e/o[r][m]   x Ci_e/o[j][m]
//   epilogue 1              u = E1 +- O1 at x = j, n-1-j; the fused update
//                           theta, residual, source q (Eqs. 12-13); q_e/o =
//                           q[j] +- q[n-1-j] -> ring of K-chunks
//   GEMM 2 (forward x, T)   Qe/o[m][r]    = Cf_e/o[m][j]  x q_e/o[r][j]
//   epilogue 2              over the row pairs: S/D[p][y'] = Q[p][r] +- Q[p][r+64]
//                           -> the owner of p (this CTA or the peer, DSMEM)
//   GEMM 3 (forward y)      R_e/o[lp][mq] = S/D[lp][y']   x Cf_e/o[mq][y']
//   epilogue 3              x K / (1 - b K) / n^2 (Eq. 21 with alpha = 0)
//                           -> ring of K-chunks
//   GEMM 4 (inverse y, T)   E4/O4[y'][lp] = Ci_e/o[y'][mq] x R'_e/o[lp][mq]
//   epilogue 4              U = E4 +- O4 at y', n-1-y' -> V_e/o of the owner of
//                           the rows (this CTA or the peer, DSMEM)
// Epilogues 1 and 3 feed GEMMs 2 and 4 chunk by chunk, so those overlap. Four
// cluster barriers per iteration order the exchanges; every CTA takes the
// same convergence decision from the same exchanged partials. Tensor memory:
// the whole 512 columns of the SM (two pairs of 128-column accumulators).
// Every mbarrier wait is bounded; after a timeout the CTA keeps its control
// flow (no early exit, so the peer never waits at a cluster barrier alone),
// stops issuing MMAs and copies, and the map reports VS_ERR_TIMEOUT.
#include <math.h>
#include <string.h>

#include <mutex>
#include <vector>

#include "vs_internal.cuh"
#include "vs_solve_common.cuh"
#include "vs_tc.cuh"

using vsk::ClusterDev;
using vsk::MapDesc;
using vsk::kFlagNonfinite;
using vsk::kFlagRunaway;
using vsk::converged;

namespace {

constexpr int kN = 256, kH = 128;
constexpr int kEpi = 256;                      // epilogue warps 0-7: lane quarter w & 3, column half w >> 2
constexpr int kThreads = kEpi + 32;            // + warp 8: copies and MMA issue
constexpr int kKc = 16;                        // K per chunk (one MMA K-step)
constexpr int kChunks = kH / kKc;              // chunks per GEMM
constexpr int kMat = kH * kKc * 2;             // one [128][16] BF16 chunk matrix: 4 KB
constexpr int kChunkBytes = 4 * kMat;          // e hi, e lo, o hi, o lo: 16 KB
constexpr int kXMat = kH * kH * 2;             // one [128][128] BF16 matrix: 32 KB
constexpr int kStages = 4;                     // constant stages
constexpr int kRing = 2;                       // epilogue -> MMA ring slots
constexpr long long kWaitLimit = 4000000LL;
constexpr int kGemmsPerIter = 4;

struct TccSlots {
  double part[2], part2[2];
  float resid[2];
  int flags[2];
};

struct alignas(1024) TccSmem {
  uint8_t x[4 * kXMat];                        // V_e hi, lo, V_o hi, lo  /  S hi, lo, D hi, lo
  uint8_t ring[kRing][kChunkBytes];
  uint8_t cst[kStages][kChunkBytes];
  uint64_t cst_full[kStages];
  uint64_t cst_empty[kStages];
  uint64_t ring_done[kRing];
  uint64_t ring_full[kRing];
  uint64_t acc;
  uint32_t tmem_base;
  uint32_t err;
  TccSlots slots;
  float red_f[kThreads / 32];
  int red_i[kThreads / 32];
  double red_d[kThreads / 32];
};

struct TccArgs {
  ClusterDev P;
  const uint8_t* cf;       // Cf_e / Cf_o in K-chunks: [chunk][e hi, e lo, o hi, o lo]
  const uint8_t* ci;       // Ci_e / Ci_o, same layout
  unsigned* err_out;       // set when a wait timed out
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
__device__ __forceinline__ void cl_sync() {
  asm volatile(
      "barrier.cluster.arrive.release.aligned;\n\t"
      "barrier.cluster.wait.acquire.aligned;" ::: "memory");
}
__device__ __forceinline__ uint32_t cl_map(const void* p, unsigned rank) {
  uint32_t a = (uint32_t)__cvta_generic_to_shared(p), r;
  asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(a), "r"(rank));
  return r;
}
__device__ __forceinline__ void st_cluster_v4(uint32_t addr, uint4 v) {
  asm volatile("st.shared::cluster.v4.b32 [%0], {%1, %2, %3, %4};" ::"r"(addr), "r"(v.x), "r"(v.y),
               "r"(v.z), "r"(v.w)
               : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, double v) {
  asm volatile("st.shared::cluster.f64 [%0], %1;" ::"r"(a), "d"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, float v) {
  asm volatile("st.shared::cluster.f32 [%0], %1;" ::"r"(a), "f"(v) : "memory");
}
__device__ __forceinline__ void st_cluster(uint32_t a, int v) {
  asm volatile("st.shared::cluster.s32 [%0], %1;" ::"r"(a), "r"(v) : "memory");
}
__device__ __forceinline__ void mbar_arrive1(uint64_t* bar) {
  asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(vstc::smem_u32(bar)) : "memory");
}
// generic-proxy shared-memory writes (local or a peer's) -> async proxy (MMA)
__device__ __forceinline__ void fence_proxy_async_all() {
  asm volatile("fence.proxy.async;" ::: "memory");
}

// 32 lanes x 16 consecutive 32-bit TMEM columns.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
      "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}
// 32 lanes x 8 consecutive columns.
__device__ __forceinline__ void tmem_ld8(uint32_t taddr, float* v) {
  uint32_t r[8];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7])
      : "r"(taddr)
      : "memory");
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 8; ++i) v[i] = __uint_as_float(r[i]);
}

// 8 consecutive K values of one row, split into BF16 hi / lo, as two 16-byte
// core-matrix rows.
__device__ __forceinline__ void split8(const float* v, uint4& hi, uint4& lo) {
  uint32_t h[4], l[4];
#pragma unroll
  for (int i = 0; i < 4; ++i) {
    __nv_bfloat16 h0, h1, l0, l1;
    vstc::split_bf16(v[2 * i], h0, l0);
    vstc::split_bf16(v[2 * i + 1], h1, l1);
    __nv_bfloat162 a = __halves2bfloat162(h0, h1), b = __halves2bfloat162(l0, l1);
    h[i] = *reinterpret_cast<uint32_t*>(&a);
    l[i] = *reinterpret_cast<uint32_t*>(&b);
  }
  hi = make_uint4(h[0], h[1], h[2], h[3]);
  lo = make_uint4(l[0], l[1], l[2], l[3]);
}

struct Pipe {
  TccSmem* sm;
  uint32_t tmem;
  int g_issue = 0;     // constant chunks whose copy was issued (MMA lane)
  int g_use = 0;       // constant chunks consumed by MMAs (MMA lane)
  int ring_uses[kRing] = {0, 0};   // epilogue: productions per slot; MMA lane: consumptions
  int ring_n = 0;      // ring chunks produced (epilogue) or consumed (MMA lane)
  int acc_n = 0;       // GEMM completions waited for (epilogue)
  bool bad = false;    // a wait timed out: stop issuing work
};

// Bounded wait by every calling thread; a timeout marks the pipe bad.
__device__ __forceinline__ bool pwait(Pipe& p, uint64_t* bar, uint32_t parity) {
  if (p.bad) return false;
  if (!vstc::mbar_wait(bar, parity, kWaitLimit)) {
    p.bad = true;
    p.sm->err = 1u;
    return false;
  }
  return true;
}

// MMA lane: issue the copy of constant chunk number g of the launch's stream
// into its stage, once the MMAs of the chunk that used the stage before are done.
__device__ __forceinline__ void issue_const(Pipe& p, const TccArgs& a, int g) {
  const int s = g % kStages;
  if (g >= kStages && !pwait(p, &p.sm->cst_empty[s], ((g - kStages) / kStages) & 1)) return;
  if (p.bad) return;
  // execution order: the first GEMM 2 (Cf), then per iteration GEMM 3 (Cf),
  // GEMM 4 (Ci), GEMM 1 (Ci), GEMM 2 (Cf)
  const int kc = g % kChunks;
  const int gemm = g < kChunks ? 3 : ((g - kChunks) / kChunks) % kGemmsPerIter;
  const uint8_t* src = (gemm == 1 || gemm == 2 ? a.ci : a.cf) + (size_t)kc * kChunkBytes;
  vstc::mbar_arrive_expect_tx(&p.sm->cst_full[s], kChunkBytes);
  vstc::bulk_g2s(p.sm->cst[s], src, kChunkBytes, &p.sm->cst_full[s]);
}

// MMA lane: keep constant copies up to kStages - 2 chunks ahead of use (the
// stage of chunk g + 2 was last used by chunk g - 2, whose MMAs are done by now).
__device__ __forceinline__ void prefetch_const(Pipe& p, const TccArgs& a) {
  while (p.g_issue < p.g_use + kStages - 1) {
    issue_const(p, a, p.g_issue);
    ++p.g_issue;
  }
}

// MMA lane: the 6 MMAs of one K-chunk into the accumulator pair at column
// `col` (e at col, o at col + 128). a_e / b_e: base addresses of the e
// operands (hi, then lo at + mat); the o operands follow at + 2 mat. sbo_*:
// the core stride of a K-major operand of K extent 128 (X) or 16 (a chunk).
__device__ __forceinline__ void mma_chunk(const Pipe& p, uint32_t col, uint32_t a_e, uint32_t a_mat,
                                          uint32_t sbo_a, uint32_t b_e, uint32_t b_mat,
                                          uint32_t sbo_b, bool accumulate) {
  const uint32_t idesc = vstc::idesc_bf16(128, 128);
#pragma unroll
  for (int eo = 0; eo < 2; ++eo) {
    const uint32_t d = p.tmem + col + 128u * eo;
    const uint32_t ah = a_e + 2u * a_mat * eo, al = ah + a_mat;
    const uint32_t bh = b_e + 2u * b_mat * eo, bl = bh + b_mat;
    const uint64_t dah = vstc::smem_desc(ah, 128, sbo_a), dal = vstc::smem_desc(al, 128, sbo_a);
    const uint64_t dbh = vstc::smem_desc(bh, 128, sbo_b), dbl = vstc::smem_desc(bl, 128, sbo_b);
    vstc::mma_bf16(d, dah, dbh, idesc, accumulate ? 1u : 0u);
    vstc::mma_bf16(d, dah, dbl, idesc, 1u);
    vstc::mma_bf16(d, dal, dbh, idesc, 1u);
  }
}

// MMA lane: a GEMM whose data operand is the X buffer (K = 128, A side) and
// whose constant streams in chunks (B side): GEMMs 1 and 3. Commits `acc`.
__device__ void gemm_x(Pipe& p, const TccArgs& a, uint32_t col) {
  const uint32_t x0 = vstc::smem_u32(p.sm->x);
  for (int kc = 0; kc < kChunks; ++kc) {
    prefetch_const(p, a);
    const int g = p.g_use, s = g % kStages;
    if (pwait(p, &p.sm->cst_full[s], (g / kStages) & 1)) {
      vstc::tc_fence_after();
      const uint32_t c0 = vstc::smem_u32(p.sm->cst[s]);
      mma_chunk(p, col, x0 + (uint32_t)kc * 256u, kXMat, (kH / 8) * 128, c0, kMat, (kKc / 8) * 128,
                kc > 0);
    }
    vstc::mma_commit(&p.sm->cst_empty[s]);
    ++p.g_use;
  }
  vstc::mma_commit(&p.sm->acc);
}

// MMA lane: a GEMM whose data operand comes chunk by chunk from the
// epilogue's ring (B side; the constant is A): GEMMs 2 and 4. Commits `acc`.
__device__ void gemm_ring(Pipe& p, const TccArgs& a, uint32_t col) {
  for (int kc = 0; kc < kChunks; ++kc) {
    prefetch_const(p, a);
    const int slot = p.ring_n % kRing;
    const bool ready = pwait(p, &p.sm->ring_full[slot], p.ring_uses[slot] & 1);
    const int g = p.g_use, s = g % kStages;
    if (ready && pwait(p, &p.sm->cst_full[s], (g / kStages) & 1)) {
      vstc::tc_fence_after();
      const uint32_t c0 = vstc::smem_u32(p.sm->cst[s]);
      const uint32_t r0 = vstc::smem_u32(p.sm->ring[slot]);
      mma_chunk(p, col, c0, kMat, (kKc / 8) * 128, r0, kMat, (kKc / 8) * 128, kc > 0);
    }
    vstc::mma_commit(&p.sm->cst_empty[s]);
    vstc::mma_commit(&p.sm->ring_done[slot]);
    ++p.g_use;
    p.ring_uses[slot]++;
    p.ring_n++;
  }
  vstc::mma_commit(&p.sm->acc);
}

// Epilogue threads: wait for the GEMM committed as number p.acc_n.
__device__ __forceinline__ void wait_acc(Pipe& p) {
  pwait(p, &p.sm->acc, p.acc_n & 1);
  ++p.acc_n;
  vstc::tc_fence_after();
}

// Epilogue threads: the ring slot of the next produced chunk, once its last
// MMAs are done.
__device__ __forceinline__ int ring_acquire(Pipe& p) {
  const int slot = p.ring_n % kRing;
  if (p.ring_uses[slot] > 0) pwait(p, &p.sm->ring_done[slot], (p.ring_uses[slot] - 1) & 1);
  return slot;
}

// Epilogue threads: a chunk written into `slot` is handed to the MMA lane.
__device__ __forceinline__ void ring_publish(Pipe& p, int slot, int t) {
  fence_proxy_async_all();
  vstc::tc_fence_before();
  asm volatile("bar.sync 1, %0;" ::"r"(kEpi) : "memory");
  if (t == 0) mbar_arrive1(&p.sm->ring_full[slot]);
  p.ring_uses[slot]++;
  p.ring_n++;
}

__device__ __forceinline__ void epi_sync() { asm volatile("bar.sync 1, %0;" ::"r"(kEpi) : "memory"); }

__global__ void __launch_bounds__(kThreads, 1) k_solve_tcc(TccArgs a) {
  extern __shared__ __align__(1024) uint8_t tcc_raw[];
  TccSmem* sm = reinterpret_cast<TccSmem*>(
      (reinterpret_cast<uintptr_t>(tcc_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const ClusterDev& P = a.P;
  const unsigned rank = cl_rank();
  const int b = __ldg(&P.order[cl_index()]);
  const MapDesc& d = P.maps[b];
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const bool mma_warp = warp == kEpi / 32;
  const int q4 = warp & 3, half = (warp >> 2) & 1;
  const int row = 32 * q4 + lane;                 // TMEM lane of this thread (epilogue)
  const float beta = P.beta, alpha = P.alpha;
  const float inv_n2 = 1.f / ((float)kN * (float)kN);

  if (t == 0) {
    for (int s = 0; s < kStages; ++s) {
      vstc::mbar_init(&sm->cst_full[s], 1);
      vstc::mbar_init(&sm->cst_empty[s], 1);
    }
    for (int s = 0; s < kRing; ++s) {
      vstc::mbar_init(&sm->ring_done[s], 1);
      vstc::mbar_init(&sm->ring_full[s], 1);
    }
    vstc::mbar_init(&sm->acc, 1);
    sm->err = 0u;
    vstc::mbar_fence_init();
  }
  if (warp == 0) vstc::tmem_alloc(&sm->tmem_base, 512);
  vstc::tc_fence_before();
  __syncthreads();
  vstc::tc_fence_after();
  Pipe p;
  p.sm = sm;
  p.tmem = sm->tmem_base;
  const uint32_t lane_base = (uint32_t)(32 * q4) << 16;

  // ---- the means of the inputs over the map (both CTAs): mu = mean P_leak0,
  // and mean P_dyn for the uniform start; compensated FP32 sums per thread
  const int y_lo = 64 * (int)rank;                // rows [y_lo, y_lo + 64) and their mirrors
  auto row_of = [&](int r) { return r < 64 ? y_lo + r : kN - 1 - (y_lo + r - 64); };
  {
    float lh = 0.f, ll = 0.f, dh = 0.f, dl = 0.f;
    auto add2 = [](float& hi, float& lo, float x) {
      const float s = hi + x, bp = s - hi;
      lo += (hi - (s - bp)) + (x - bp);
      hi = s;
    };
    for (int i = t; i < 128 * kN / 4; i += kThreads) {
      const int r = i / (kN / 4), x4 = i % (kN / 4);
      const size_t idx = (size_t)row_of(r) * kN + 4 * x4;
      const float4 l4 = __ldg(reinterpret_cast<const float4*>(d.p_leak0 + idx));
      const float4 p4 = __ldg(reinterpret_cast<const float4*>(d.p_dyn + idx));
      add2(lh, ll, l4.x); add2(lh, ll, l4.y); add2(lh, ll, l4.z); add2(lh, ll, l4.w);
      add2(dh, dl, p4.x); add2(dh, dl, p4.y); add2(dh, dl, p4.z); add2(dh, dl, p4.w);
    }
    double tl = (double)lh + (double)ll, td = (double)dh + (double)dl;
    tl = vsk::block_sum(tl, sm->red_d);
    td = vsk::block_sum(td, sm->red_d);
    if (t == 0) {
      for (unsigned r = 0; r < 2; ++r) {
        st_cluster(cl_map(&sm->slots.part[rank], r), tl);
        st_cluster(cl_map(&sm->slots.part2[rank], r), td);
      }
    }
  }
  cl_sync();
  const double mu = (sm->slots.part[0] + sm->slots.part[1]) / ((double)kN * kN);
  int status = VS_OK, iters = 0, growth = 0;
  float prev = INFINITY, th0 = 0.f, mu_p = (float)mu;
  bool stop = false;
  if ((double)beta * mu * (double)d.kmax >= 0.999) {
    status = VS_ERR_RUNAWAY;
    stop = true;
  } else {
    // uniform mode of the die (a scalar fixed point) as the start, and the
    // preconditioner mu_p = mu (1 + 2 alpha u) (as the FP32 engines)
    const float pdm = (float)((sm->slots.part2[0] + sm->slots.part2[1]) / ((double)kN * kN));
    const float muf = (float)mu, k00 = __ldg(d.Kt);
    float ub = 0.f;
    bool ok = true;
    for (int k = 0; k < 16 && ok; ++k) {
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
  }
  const float bm = beta * mu_p;

  // ---- epilogue 1 / first source: 8 x-positions j0 .. j0 + 7 of this
  // thread's row and their mirrors n-1-j per chunk. The global inputs of a
  // chunk are loaded one chunk ahead.
  struct RowIn {
    float pl[16], pd[16], sk[16], old[16];
  };
  float resid = 0.f;
  int flags = 0;
  auto load_row = [&](int kc, bool with_old, RowIn& in) {
    const int j0 = kc * kKc + 8 * half;
    const size_t ia = (size_t)row_of(row) * kN + j0, ib = (size_t)row_of(row) * kN + (kN - 8 - j0);
    auto ld8 = [&](const float* src, float* dst, bool ro) {
      float4 a0, a1, b0, b1;
      if (ro) {
        a0 = __ldg(reinterpret_cast<const float4*>(src + ia));
        a1 = __ldg(reinterpret_cast<const float4*>(src + ia + 4));
        b0 = __ldg(reinterpret_cast<const float4*>(src + ib));
        b1 = __ldg(reinterpret_cast<const float4*>(src + ib + 4));
      } else {
        a0 = *reinterpret_cast<const float4*>(src + ia);
        a1 = *reinterpret_cast<const float4*>(src + ia + 4);
        b0 = *reinterpret_cast<const float4*>(src + ib);
        b1 = *reinterpret_cast<const float4*>(src + ib + 4);
      }
      // dst[i] at x = j0 + i, dst[8 + i] at x = n-1-(j0+i) (= ib + 7 - i)
      dst[0] = a0.x; dst[1] = a0.y; dst[2] = a0.z; dst[3] = a0.w;
      dst[4] = a1.x; dst[5] = a1.y; dst[6] = a1.z; dst[7] = a1.w;
      dst[15] = b0.x; dst[14] = b0.y; dst[13] = b0.z; dst[12] = b0.w;
      dst[11] = b1.x; dst[10] = b1.y; dst[9] = b1.z; dst[8] = b1.w;
    };
    ld8(d.p_leak0, in.pl, true);
    ld8(d.p_dyn, in.pd, true);
    if (d.s) {
      ld8(d.s, in.sk, true);
    } else {
#pragma unroll
      for (int i = 0; i < 16; ++i) in.sk[i] = 1.f;
    }
    if (with_old) ld8(d.theta, in.old, false);
  };
  auto source_chunk = [&](int kc, int slot, bool first, bool have_old, const RowIn& in) {
    const int j0 = kc * kKc + 8 * half;
    const size_t ia = (size_t)row_of(row) * kN + j0, ib = (size_t)row_of(row) * kN + (kN - 8 - j0);
    float e[8], o[8];
    if (!first) {
      tmem_ld8(p.tmem + lane_base + (uint32_t)j0, e);
      tmem_ld8(p.tmem + lane_base + 128u + (uint32_t)j0, o);
    }
    // theta = phi(u) (Eq. 12), residual against the previous iterate, and the
    // preconditioned source q = P_dyn + P_leak0 + beta P_leak0 theta - b u
    // (b = beta mu_p, Sec. IV-C) of the next transform
    float th[16], q[16];
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      float uu;
      if (first) {
        th[i] = th0;
        uu = __fdividef(th0, in.sk[i] * fmaf(alpha, th0, 1.f));
      } else {
        const int k = i & 7;
        uu = i < 8 ? e[k] + o[k] : e[k] - o[k];
        const float den = fmaf(-alpha * in.sk[i], uu, 1.f);
        if (!(den > 0.05f)) flags |= kFlagRunaway;
        th[i] = __fdividef(in.sk[i] * uu, den);
        const float pv = have_old ? in.old[i] : th0;
        if (!isfinite(th[i])) flags |= kFlagNonfinite;
        else resid = fmaxf(resid, fabsf(th[i] - pv));
      }
      q[i] = fmaf(beta * in.pl[i], th[i], in.pd[i] + in.pl[i]) - bm * uu;
    }
    if (!first) {
      *reinterpret_cast<float4*>(d.theta + ia) = make_float4(th[0], th[1], th[2], th[3]);
      *reinterpret_cast<float4*>(d.theta + ia + 4) = make_float4(th[4], th[5], th[6], th[7]);
      *reinterpret_cast<float4*>(d.theta + ib) = make_float4(th[15], th[14], th[13], th[12]);
      *reinterpret_cast<float4*>(d.theta + ib + 4) = make_float4(th[11], th[10], th[9], th[8]);
    }
    float qe[8], qo[8];
#pragma unroll
    for (int i = 0; i < 8; ++i) {
      qe[i] = q[i] + q[8 + i];
      qo[i] = q[i] - q[8 + i];
    }
    uint4 h, l;
    uint8_t* base = sm->ring[slot];
    const uint32_t off = vstc::core_off(row, 8 * half, kKc);
    split8(qe, h, l);
    *reinterpret_cast<uint4*>(base + off) = h;
    *reinterpret_cast<uint4*>(base + kMat + off) = l;
    split8(qo, h, l);
    *reinterpret_cast<uint4*>(base + 2 * kMat + off) = h;
    *reinterpret_cast<uint4*>(base + 3 * kMat + off) = l;
  };

  // epilogue 1 (or the first source) feeding GEMM 2 chunk by chunk
  auto phase_rows = [&](bool first) {
    const bool have_old = !first && iters > 1;   // iterate 1 compares with the uniform start
    RowIn ra, rb;                                  // two chunks in flight, static indices
    load_row(0, have_old, ra);
#pragma unroll 1
    for (int kc = 0; kc < kChunks; kc += 2) {
      load_row(kc + 1, have_old, rb);
      int slot = ring_acquire(p);
      source_chunk(kc, slot, first, have_old, ra);
      ring_publish(p, slot, t);
      if (kc + 2 < kChunks) load_row(kc + 2, have_old, ra);
      slot = ring_acquire(p);
      source_chunk(kc + 1, slot, first, have_old, rb);
      ring_publish(p, slot, t);
    }
  };

  // epilogue 2: Q[p][r] (lane = m, p = 2m + eo) summed / differenced over the
  // row pairs -> S / D rows lp = p - 128 c' of the owner c' (K index y')
  auto epilogue2 = [&]() {
    const int m = row;
    const unsigned dst = (unsigned)(m >> 6);                    // owner of p = 2m, 2m + 1
    const uint32_t xr = cl_map(sm->x, dst);
#pragma unroll 1
    for (int eo = 0; eo < 2; ++eo) {
      const int lp = 2 * m + eo - 128 * (int)dst;
      const uint32_t col = 256u + 128u * eo;
      float a0[32], a1[32];
      tmem_ld16(p.tmem + lane_base + col + 32u * half, a0);
      tmem_ld16(p.tmem + lane_base + col + 32u * half + 16u, a0 + 16);
      tmem_ld16(p.tmem + lane_base + col + 64u + 32u * half, a1);
      tmem_ld16(p.tmem + lane_base + col + 64u + 32u * half + 16u, a1 + 16);
#pragma unroll
      for (int g = 0; g < 4; ++g) {
        float sv[8], dv[8];
#pragma unroll
        for (int i = 0; i < 8; ++i) {
          sv[i] = a0[8 * g + i] + a1[8 * g + i];
          dv[i] = a0[8 * g + i] - a1[8 * g + i];
        }
        const int yk = 64 * (int)rank + 32 * half + 8 * g;      // K index y'
        const uint32_t off = vstc::core_off(lp, yk, kH);
        uint4 h, l;
        split8(sv, h, l);
        st_cluster_v4(xr + off, h);
        st_cluster_v4(xr + kXMat + off, l);
        split8(dv, h, l);
        st_cluster_v4(xr + 2 * kXMat + off, h);
        st_cluster_v4(xr + 3 * kXMat + off, l);
      }
    }
  };

  // epilogue 3 feeding GEMM 4: R (lane lp, column mq) times the multiplier
  // K / (1 - b K) / n^2 at (p, q = 2 mq + eo); K loaded one chunk ahead
  auto phase_cols = [&]() {
    const int lp = row, pidx = 128 * (int)rank + lp;
    auto load_k = [&](int kc, float* dst) {
      const float4* kr = reinterpret_cast<const float4*>(d.Kt + (size_t)pidx * kN + 2 * (kc * kKc + 8 * half));
#pragma unroll
      for (int i = 0; i < 4; ++i) {
        const float4 v = __ldg(kr + i);
        dst[4 * i] = v.x; dst[4 * i + 1] = v.y; dst[4 * i + 2] = v.z; dst[4 * i + 3] = v.w;
      }
    };
    auto cols_chunk = [&](int kc, const float* kk) {
      const int slot = ring_acquire(p);
      const int m0 = kc * kKc + 8 * half;
      float re[8], ro[8];
      tmem_ld8(p.tmem + lane_base + (uint32_t)m0, re);
      tmem_ld8(p.tmem + lane_base + 128u + (uint32_t)m0, ro);
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        const float ke = kk[2 * i], ko = kk[2 * i + 1];
        re[i] *= __fdividef(ke, 1.f - bm * ke) * inv_n2;
        ro[i] *= __fdividef(ko, 1.f - bm * ko) * inv_n2;
      }
      uint4 h, l;
      uint8_t* base = sm->ring[slot];
      const uint32_t off = vstc::core_off(lp, 8 * half, kKc);
      split8(re, h, l);
      *reinterpret_cast<uint4*>(base + off) = h;
      *reinterpret_cast<uint4*>(base + kMat + off) = l;
      split8(ro, h, l);
      *reinterpret_cast<uint4*>(base + 2 * kMat + off) = h;
      *reinterpret_cast<uint4*>(base + 3 * kMat + off) = l;
      ring_publish(p, slot, t);
    };
    float ka[16], kb[16];                          // two chunks in flight, static indices
    load_k(0, ka);
#pragma unroll 1
    for (int kc = 0; kc < kChunks; kc += 2) {
      load_k(kc + 1, kb);
      cols_chunk(kc, ka);
      if (kc + 2 < kChunks) load_k(kc + 2, ka);
      cols_chunk(kc + 1, kb);
    }
  };

  // epilogue 4: U = E4 +- O4 at rows y' (lane) and n-1-y' -> V_e / V_o rows
  // r, r + 64 of the owner of the rows (K index m = p / 2)
  auto epilogue4 = [&]() {
    const int yp = row;
    const unsigned dst = (unsigned)(yp >> 6);
    const int r = yp - 64 * (int)dst;
    const uint32_t xr = cl_map(sm->x, dst);
#pragma unroll 1
    for (int c4 = 0; c4 < 4; ++c4) {
      const uint32_t c0 = (uint32_t)(64 * half + 16 * c4);      // lp chunk of 16
      float ev[16], ov[16];
      tmem_ld16(p.tmem + lane_base + 256u + c0, ev);
      tmem_ld16(p.tmem + lane_base + 384u + c0, ov);
      float ue[8], uo[8], me[8], mo[8];
#pragma unroll
      for (int i = 0; i < 8; ++i) {
        ue[i] = ev[2 * i] + ov[2 * i];          // row y', even p
        uo[i] = ev[2 * i + 1] + ov[2 * i + 1];  // row y', odd p
        me[i] = ev[2 * i] - ov[2 * i];          // mirror row, even p
        mo[i] = ev[2 * i + 1] - ov[2 * i + 1];
      }
      const int mk = 64 * (int)rank + (int)c0 / 2;                // K index m of lp = c0
      uint4 h, l;
      const uint32_t o0 = vstc::core_off(r, mk, kH), o1 = vstc::core_off(r + 64, mk, kH);
      split8(ue, h, l);
      st_cluster_v4(xr + o0, h);
      st_cluster_v4(xr + kXMat + o0, l);
      split8(uo, h, l);
      st_cluster_v4(xr + 2 * kXMat + o0, h);
      st_cluster_v4(xr + 3 * kXMat + o0, l);
      split8(me, h, l);
      st_cluster_v4(xr + o1, h);
      st_cluster_v4(xr + kXMat + o1, l);
      split8(mo, h, l);
      st_cluster_v4(xr + 2 * kXMat + o1, h);
      st_cluster_v4(xr + 3 * kXMat + o1, l);
    }
  };

  // the convergence decision of iterate `it`, identical in both CTAs
  auto decide = [&](int it) {
    const float rr = fmaxf(sm->slots.resid[0], sm->slots.resid[1]);
    const int ff = sm->slots.flags[0] | sm->slots.flags[1];
    iters = it;
    if (ff & 4) {
      status = VS_ERR_TIMEOUT;
      stop = true;
    } else if (ff & kFlagNonfinite) {
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
  auto cluster_barrier = [&]() {
    vstc::tc_fence_before();
    cl_sync();
    vstc::tc_fence_after();
  };

  if (!stop) {
    if (mma_warp) {
      // ---- the MMA warp: lane 0 issues copies and MMAs; the whole warp takes
      // part in the cluster barriers, in the epilogue's order
      if (lane == 0) gemm_ring(p, a, 256u);                 // first GEMM 2
      __syncwarp();
      for (int it = 0;; ++it) {
        cluster_barrier();                                  // B1
        if (it >= 1) {
          decide(it);
          if (stop) break;
        }
        cluster_barrier();                                  // B3
        if (lane == 0) {
          gemm_x(p, a, 0u);                                 // GEMM 3 -> R_e / R_o
          gemm_ring(p, a, 256u);                            // GEMM 4 <- epilogue 3
        }
        __syncwarp();
        cluster_barrier();                                  // B2
        cluster_barrier();                                  // B4
        if (lane == 0) {
          gemm_x(p, a, 0u);                                 // GEMM 1 -> E1 / O1
          gemm_ring(p, a, 256u);                            // GEMM 2 <- epilogue 1
        }
        __syncwarp();
      }
      // constant copies issued ahead of use must land before the CTA exits
      if (lane == 0)
        for (int g = p.g_use; g < p.g_issue; ++g)
          pwait(p, &sm->cst_full[g % kStages], (g / kStages) & 1);
      __syncwarp();
    } else {
      // ---- the epilogue warps
      phase_rows(true);                                     // first source -> GEMM 2
      for (int it = 0;; ++it) {
        wait_acc(p);                                        // GEMM 2 done
        if (it >= 1) {
          // residual and flags of iterate `it` to both CTAs
          float rm = resid;
          int fo = flags;
#pragma unroll
          for (int o = 16; o > 0; o >>= 1) {
            rm = fmaxf(rm, __shfl_down_sync(0xffffffffu, rm, o));
            fo |= __shfl_down_sync(0xffffffffu, fo, o);
          }
          if (lane == 0) {
            sm->red_f[warp] = rm;
            sm->red_i[warp] = fo;
          }
          epi_sync();
          if (t == 0) {
            rm = 0.f;
            fo = 0;
            for (int w = 0; w < kEpi / 32; ++w) {
              rm = fmaxf(rm, sm->red_f[w]);
              fo |= sm->red_i[w];
            }
            if (sm->err) fo |= 4;
            for (unsigned rr = 0; rr < 2; ++rr) {
              st_cluster(cl_map(&sm->slots.resid[rank], rr), rm);
              st_cluster(cl_map(&sm->slots.flags[rank], rr), fo);
            }
          }
        }
        cluster_barrier();                                  // B1
        if (it >= 1) {
          decide(it);
          resid = 0.f;
          flags = 0;
          if (stop) break;
        }
        epilogue2();
        fence_proxy_async_all();
        cluster_barrier();                                  // B3: S / D complete in both CTAs
        wait_acc(p);                                        // GEMM 3 done
        phase_cols();                                       // epilogue 3 + GEMM 4
        wait_acc(p);                                        // GEMM 4 (and 3) done
        cluster_barrier();                                  // B2: the peer's GEMM 3 is done with X
        epilogue4();
        fence_proxy_async_all();
        cluster_barrier();                                  // B4: V complete in both CTAs
        wait_acc(p);                                        // GEMM 1 done
        iters = it + 1;
        phase_rows(false);                                  // epilogue 1 + GEMM 2
      }
    }
  }
  vstc::tc_fence_before();
  __syncthreads();
  if (warp == 0) vstc::tmem_dealloc(p.tmem, 512);
  if (rank == 0 && t == 0) {
    vs_solve_info* inf = P.info + b;
    inf->status = status;
    inf->iterations = iters;
    inf->residual_K = (double)prev;
    inf->mu_W = mu;
    inf->fell_back = 0;
  }
  if (t == 0 && sm->err) atomicOr(a.err_out, 1u);
  cl_sync();                                  // no CTA leaves while its peer may store into it
}

// Host: the constant matrices, BF16 hi/lo, K-chunks of 16 in core-matrix order.
uint16_t bf16_bits(double x) {
  float f = (float)x;
  uint32_t u;
  memcpy(&u, &f, 4);
  u += 0x7FFFu + ((u >> 16) & 1u);
  return (uint16_t)(u >> 16);
}
double bf16_value(uint16_t h) {
  uint32_t u = (uint32_t)h << 16;
  float f;
  memcpy(&f, &u, 4);
  return (double)f;
}

// fwd: rows m (frequency), K = j (position): e = C[2m][j], o = C[2m+1][j].
// inv: rows j (position), K = m (frequency): e = w_2m C[2m][j], o = 2 C[2m+1][j].
std::vector<uint8_t> tile_pair(bool inverse) {
  const double pi = 3.141592653589793238462643383279502884;
  std::vector<uint8_t> out((size_t)kChunks * kChunkBytes, 0);
  for (int rr = 0; rr < kH; ++rr)
    for (int k = 0; k < kH; ++k)
      for (int eo = 0; eo < 2; ++eo) {
        const int m = inverse ? k : rr, j = inverse ? rr : k;
        const int freq = 2 * m + eo;
        double v = cos(pi * freq * (2.0 * j + 1.0) / (2.0 * kN));
        if (inverse) v *= (freq == 0 ? 1.0 : 2.0);
        const uint16_t hi = bf16_bits(v), lo = bf16_bits(v - bf16_value(hi));
        const int kc = k / kKc;
        const size_t base = (size_t)kc * kChunkBytes + (size_t)eo * 2 * kMat +
                            vstc::core_off(rr, k % kKc, kKc);
        memcpy(&out[base], &hi, 2);
        memcpy(&out[base + kMat], &lo, 2);
      }
  return out;
}

struct TccMats {
  uint8_t* cf = nullptr;
  uint8_t* ci = nullptr;
  unsigned* err = nullptr;
};
std::mutex g_tcc_mutex;
std::vector<std::pair<int, TccMats>> g_tcc;     // per device
bool g_tcc_attr[64] = {};

const TccMats* tcc_mats(int* status) {
  int dev = 0;
  cudaGetDevice(&dev);
  std::lock_guard<std::mutex> lk(g_tcc_mutex);
  for (auto& e : g_tcc)
    if (e.first == dev) return &e.second;
  TccMats m;
  std::vector<uint8_t> f = tile_pair(false), iv = tile_pair(true);
  cudaError_t e = cudaMalloc(&m.cf, f.size());
  if (e == cudaSuccess) e = cudaMalloc(&m.ci, iv.size());
  if (e == cudaSuccess) e = cudaMalloc(&m.err, sizeof(unsigned));
  if (e == cudaSuccess) e = cudaMemcpy(m.cf, f.data(), f.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(m.ci, iv.data(), iv.size(), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(m.err, 0, sizeof(unsigned));
  if (e != cudaSuccess) {
    cudaFree(m.cf);
    cudaFree(m.ci);
    cudaFree(m.err);
    *status = vs_set_error(e == cudaErrorMemoryAllocation ? VS_ERR_OOM : VS_ERR_CUDA,
                           "tensor-core cluster matrices: %s", cudaGetErrorString(e));
    return nullptr;
  }
  g_tcc.push_back({dev, m});
  return &g_tcc.back().second;
}

static_assert(sizeof(TccSmem) + 1024 <= 232448, "shared memory of the tensor-core cluster engine");

}  // namespace

size_t vs_tcc_smem() { return sizeof(TccSmem) + 1024; }

bool vs_tcc_ok(int n) { return n == kN; }

// VS_OK if at least one pair of CTAs of the engine fits on the device.
int vs_tcc_check(cudaStream_t s) {
  int dev = 0;
  VS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !g_tcc_attr[dev]) {
    VS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_solve_tcc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)vs_tcc_smem()));
    g_tcc_attr[dev] = true;
  }
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = vs_tcc_smem();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  int clusters = 0;
  VS_CUDA_TRY(cudaOccupancyMaxActiveClusters(&clusters, (const void*)k_solve_tcc, &cfg));
  if (clusters < 1) return vs_set_error(VS_ERR_INVALID_ARG, "no CTA pair of the tensor-core cluster engine fits");
  int st = VS_OK;
  if (!tcc_mats(&st)) return st;
  return VS_OK;
}

// Launch of the engine over `count` maps (cluster index -> map via P.order).
int vs_tcc_launch(const ClusterDev& P, int count, cudaStream_t s) {
  int st = VS_OK;
  const TccMats* m = tcc_mats(&st);
  if (!m) return st;
  int dev = 0;
  VS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev >= 0 && dev < 64 && !g_tcc_attr[dev]) {
    VS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_solve_tcc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)vs_tcc_smem()));
    g_tcc_attr[dev] = true;
  }
  TccArgs a;
  a.P = P;
  a.cf = m->cf;
  a.ci = m->ci;
  a.err_out = m->err;
  cudaLaunchConfig_t cfg = {};
  cfg.gridDim = dim3(2u * (unsigned)count);
  cfg.blockDim = dim3(kThreads);
  cfg.dynamicSmemBytes = vs_tcc_smem();
  cfg.stream = s;
  cudaLaunchAttribute attr[1];
  attr[0].id = cudaLaunchAttributeClusterDimension;
  attr[0].val.clusterDim.x = 2;
  attr[0].val.clusterDim.y = 1;
  attr[0].val.clusterDim.z = 1;
  cfg.attrs = attr;
  cfg.numAttrs = 1;
  cudaError_t e = cudaLaunchKernelEx(&cfg, k_solve_tcc, a);
  if (e != cudaSuccess)
    return vs_set_error(VS_ERR_CUDA, "tensor-core cluster launch: %s", cudaGetErrorString(e));
  return VS_OK;
}
