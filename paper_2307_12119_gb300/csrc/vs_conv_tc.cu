// 3x3 convolution (zero padding) of the warm-start network as a tcgen05
// implicit GEMM, for inference:
//   out[b][co][p] = bias[co] + sum_{ci, ky, kx} W[co][ci][ky][kx] in[b][ci][p + (ky-1, kx-1)]
// is D[m][n] = sum_k A[m][k] B[n][k] with m = a tile of 128 output pixels of one
// image, n = co (padded to a multiple of 16), k = r * cp + ci with r = 3 ky + kx
// the tap and cp = cin rounded up to a multiple of 8 (padded to a multiple of
// 64): every 8 consecutive k share one tap, so a thread gathers 8 channels at
// one neighbouring pixel with one bounds check. A (im2col of the FP32 activations, rounded to BF16) is
// built by the CTA's threads in shared memory, 64 k at a time into two
// alternating stages; B (the model's BF16 weights) is staged once per CTA; the
// FP32 accumulator lives in tensor memory and the epilogue adds the bias,
// applies ReLU and stores FP32 NCHW. One elected thread issues the MMAs
// (kind::f16, BF16 x BF16 -> FP32). Persistent CTAs loop over the tiles.
// Waits are bounded; a timeout stops the launch's MMAs and is reported.
#include <cuda_bf16.h>
#include <stdint.h>

#include "vs_internal.cuh"
#include "vs_tc.cuh"

namespace {

constexpr int kThreads = 256;
constexpr int kM = 128;                       // output pixels per tile
constexpr int kKc = 64;                       // k per A stage
constexpr int kAStage = kM * kKc * 2;         // 16 KB
constexpr int kMaxW = 64 * 1024;              // staged weights at most (bytes)
constexpr long long kWaitLimit = 4000000LL;

struct ConvSmem {
  uint8_t a[2][kAStage];
  uint8_t w[kMaxW];
  uint64_t done[2];
  uint64_t acc;
  uint32_t tmem_base;
  uint32_t err;
};

struct ConvArgs {
  const float* in;
  int in_ctot, cin;
  const __nv_bfloat16* W;
  const float* bias;
  float* out;
  int out_ctot, cout;
  int B, H, relu;
  int np, kp, cp;                             // padded N, K and channels per tap
  unsigned* err;
};

__global__ void __launch_bounds__(kThreads, 2) k_conv_tc(ConvArgs a) {
  extern __shared__ __align__(1024) uint8_t conv_raw[];
  ConvSmem* sm = reinterpret_cast<ConvSmem*>(
      (reinterpret_cast<uintptr_t>(conv_raw) + 1023) & ~static_cast<uintptr_t>(1023));
  const int t = threadIdx.x, lane = t & 31, warp = t >> 5;
  const int H = a.H, HW = H * H, cp = a.cp;
  const int nkc = a.kp / kKc;
  if (t == 0) {
    vstc::mbar_init(&sm->done[0], 1);
    vstc::mbar_init(&sm->done[1], 1);
    vstc::mbar_init(&sm->acc, 1);
    sm->err = 0u;
    vstc::mbar_fence_init();
  }
  // weights [np][kp] K-major in core-matrix order, k = r * cp + ci, zero padded
  for (int i = t; i < a.np * (a.kp / 8); i += kThreads) {
    const int n = i / (a.kp / 8), k0 = (i % (a.kp / 8)) * 8;
    const int r = k0 / cp, ci0 = k0 - r * cp;
    uint32_t wv[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      __nv_bfloat16 lo = __float2bfloat16(0.f), hi = __float2bfloat16(0.f);
      const int ca = ci0 + 2 * j, cb = ca + 1;
      if (n < a.cout && r < 9 && ca < a.cin) lo = a.W[((size_t)n * a.cin + ca) * 9 + r];
      if (n < a.cout && r < 9 && cb < a.cin) hi = a.W[((size_t)n * a.cin + cb) * 9 + r];
      __nv_bfloat162 p = __halves2bfloat162(lo, hi);
      wv[j] = *reinterpret_cast<uint32_t*>(&p);
    }
    *reinterpret_cast<uint4*>(sm->w + vstc::core_off(n, k0, a.kp)) = make_uint4(wv[0], wv[1], wv[2], wv[3]);
  }
  if (warp == 0) vstc::tmem_alloc(&sm->tmem_base, 32);
  vstc::fence_proxy_async_smem();
  vstc::tc_fence_before();
  __syncthreads();
  vstc::tc_fence_after();
  const uint32_t tmem = sm->tmem_base;
  const uint32_t idesc = vstc::idesc_bf16(kM, a.np);
  const uint32_t sbo_a = (kKc / 8) * 128, sbo_w = (uint32_t)(a.kp / 8) * 128;
  const int tiles = a.B * HW / kM;
  int uses[2] = {0, 0}, accs = 0;
  bool bad = false;
  auto wait = [&](uint64_t* bar, uint32_t par) {
    if (bad) return false;
    if (!vstc::mbar_wait(bar, par, kWaitLimit)) {
      bad = true;
      sm->err = 1u;
    }
    return !bad;
  };
  for (int tile = blockIdx.x; tile < tiles; tile += gridDim.x) {
    const int pix0 = tile * kM, b = pix0 / HW, p0 = pix0 % HW;
    const float* ib = a.in + (size_t)b * a.in_ctot * HW;
    for (int c = 0; c < nkc; ++c) {
      const int s = c & 1;
      if (uses[s] > 0) wait(&sm->done[s], (uses[s] - 1) & 1);
      // im2col of k in [c kKc, (c+1) kKc): item i -> pixel m = i % 128, octet
      // i / 128 = 8 channels ci0 .. ci0 + 7 at tap r
      for (int i = t; i < kM * (kKc / 8); i += kThreads) {
        const int m = i % kM, oct = i / kM;
        const int p = p0 + m, y = p / H, x = p % H;
        const int k0 = c * kKc + oct * 8, r = k0 / cp, ci0 = k0 - r * cp;
        const int yy = y + r / 3 - 1, xx = x + r % 3 - 1;
        const bool in_img = r < 9 && yy >= 0 && yy < H && xx >= 0 && xx < H;
        const float* src = ib + (size_t)ci0 * HW + (in_img ? yy * H + xx : 0);
        float v[8];
#pragma unroll
        for (int j = 0; j < 8; ++j) v[j] = (in_img && ci0 + j < a.cin) ? __ldg(src + (size_t)j * HW) : 0.f;
        uint32_t pk[4];
#pragma unroll
        for (int j = 0; j < 4; ++j) {
          __nv_bfloat162 q = __floats2bfloat162_rn(v[2 * j], v[2 * j + 1]);
          pk[j] = *reinterpret_cast<uint32_t*>(&q);
        }
        *reinterpret_cast<uint4*>(sm->a[s] + vstc::core_off(m, oct * 8, kKc)) =
            make_uint4(pk[0], pk[1], pk[2], pk[3]);
      }
      vstc::fence_proxy_async_smem();
      vstc::tc_fence_before();
      __syncthreads();
      if (t == 0) {
        vstc::tc_fence_after();
        if (!bad) {
          const uint32_t a0 = vstc::smem_u32(sm->a[s]), w0 = vstc::smem_u32(sm->w);
#pragma unroll
          for (int ks = 0; ks < kKc / 16; ++ks) {
            const uint64_t da = vstc::smem_desc(a0 + ks * 256, 128, sbo_a);
            const uint64_t dw = vstc::smem_desc(w0 + (uint32_t)(c * (kKc / 8) + 2 * ks) * 128, 128, sbo_w);
            vstc::mma_bf16(tmem, da, dw, idesc, (c > 0 || ks > 0) ? 1u : 0u);
          }
        }
        vstc::mma_commit(&sm->done[s]);
        if (c == nkc - 1) vstc::mma_commit(&sm->acc);
      }
      uses[s]++;
    }
    // epilogue: warps 0-3 (lanes = pixels), bias, ReLU, FP32 NCHW stores
    wait(&sm->acc, accs & 1);
    ++accs;
    vstc::tc_fence_after();
    if (warp < 4) {
      const int m = 32 * warp + lane, p = p0 + m;
      float* ob = a.out + (size_t)b * a.out_ctot * HW;
      for (int c0 = 0; c0 < a.np; c0 += 16) {
        uint32_t r[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
            "{%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];"
            : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
              "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]),
              "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
            : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)c0)
            : "memory");
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int co = c0 + j;
          if (co < a.cout) {
            const float v = __uint_as_float(r[j]) + __ldg(&a.bias[co]);
            ob[(size_t)co * HW + p] = a.relu ? fmaxf(v, 0.f) : v;
          }
        }
      }
    }
    vstc::tc_fence_before();
    __syncthreads();                    // TMEM read before the next tile's MMAs
  }
  // every MMA of this CTA is complete (the last wait was on its last tile)
  __syncthreads();
  if (warp == 0) vstc::tmem_dealloc(tmem, 32);
  if (t == 0 && sm->err) atomicOr(a.err, 1u);
}

unsigned* g_conv_err[64] = {};
bool g_conv_attr[64] = {};

}  // namespace

// Runs one layer on the tensor cores; -1 when the layer's shape does not fit
// this kernel (the caller then uses the SIMT convolution).
int vs_conv_tc(const float* in, int in_ctot, int cin, const void* W, const float* bias,
               float* out, int out_ctot, int cout, int B, int H, int relu, cudaStream_t s) {
  const int cp = (cin + 7) / 8 * 8;
  const int np = (cout + 15) / 16 * 16, kp = (cp * 9 + kKc - 1) / kKc * kKc;
  if (np > 256 || (size_t)np * kp * 2 > (size_t)kMaxW || (H * H) % kM) return -1;
  int dev = 0, sms = 0;
  VS_CUDA_TRY(cudaGetDevice(&dev));
  if (dev < 0 || dev >= 64) return -1;
  if (!g_conv_err[dev]) {
    VS_CUDA_TRY(cudaMalloc(&g_conv_err[dev], sizeof(unsigned)));
    VS_CUDA_TRY(cudaMemset(g_conv_err[dev], 0, sizeof(unsigned)));
  }
  const size_t smem = sizeof(ConvSmem) + 1024;
  if (!g_conv_attr[dev]) {
    VS_CUDA_TRY(cudaFuncSetAttribute((const void*)k_conv_tc, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                     (int)smem));
    g_conv_attr[dev] = true;
  }
  VS_CUDA_TRY(cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev));
  ConvArgs a = {in, in_ctot, cin, static_cast<const __nv_bfloat16*>(W), bias, out, out_ctot, cout,
                B, H, relu, np, kp, cp, g_conv_err[dev]};
  const int tiles = B * H * H / kM;
  k_conv_tc<<<tiles < 2 * sms ? tiles : 2 * sms, kThreads, smem, s>>>(a);
  VS_CUDA_TRY(cudaGetLastError());
  return VS_OK;
}
