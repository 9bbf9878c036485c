// Learned warm start of the leakage/conductivity fixed point.
//
// A small U-Net maps reduced-resolution features of the first iterate of a
// solve to the remaining correction of the temperature:
//   features (R x R, averaged over blocks of n/R cells):
//     f0 = theta_1 / 100            first iterate of the fixed point [K/100]
//     f1 = 10 (P_leak0 / mean - 1)  leakage variation
//     f2 = 30 (s - 1)               conductivity variation
//   target: (theta* - theta_1) / 10 averaged the same way.
// The prediction, upsampled bilinearly, gives theta_init = theta_1 + 10 y for
// the warm-started solve (vs_batch_item.theta_init); the solve itself decides
// convergence, so a poor prediction costs iterations, never accuracy.
//
// Network (C = base channels, ReLU after every conv but the last):
//   x[3,R] -> conv C -> conv C (=s1) -> pool -> conv 2C -> conv 2C (=s2) -> pool
//   -> conv 2C -> up, concat s2 -> conv C -> up, concat s1 -> conv C -> conv 1
// Weights are BF16 (FP32 master copy in the optimiser), activations and
// accumulation FP32; every layer is a 3x3 convolution with zero padding.
// Training (forward and backward) runs these SIMT kernels; inference in the
// warm plan runs the convolutions as tcgen05 implicit GEMMs (vs_conv_tc.cu,
// BF16 activations) where a layer's shape fits.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>
#include <string.h>

#include <cuda_bf16.h>

#include <algorithm>
#include <utility>
#include <vector>

#include "vs_internal.cuh"

namespace {

constexpr int kLayers = 8;

struct TView {       // a channel slice of an NCHW tensor
  float* p;          // element (b=0, c=c_off, 0, 0)
  int ctot;          // channels of the underlying tensor (batch stride = ctot*H*W)
};

// ------------------------------------------------------------ kernels

// out[b][co][y][x] = bias[co] + sum_ci,ky,kx W[co][ci][ky][kx] in[b][ci][y+ky-1][x+kx-1]
// One thread per (b, 4 output channels, y, x).
__global__ void k_conv_fwd(const float* __restrict__ in, int in_ctot, int cin,
                           const __nv_bfloat16* __restrict__ W, const float* __restrict__ bias,
                           float* __restrict__ out, int out_ctot, int cout, int B, int H, int relu) {
  const int HW = H * H;
  const int cg = (cout + 3) / 4;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)B * cg * HW;
  if (t >= total) return;
  int pix = (int)(t % HW);
  int g = (int)((t / HW) % cg);
  int b = (int)(t / ((long long)HW * cg));
  int y = pix / H, x = pix % H;
  float acc[4];
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int co = 4 * g + j;
    acc[j] = co < cout ? bias[co] : 0.f;
  }
  const float* ib = in + (size_t)b * in_ctot * HW;
  for (int ci = 0; ci < cin; ++ci) {
    const float* ic = ib + (size_t)ci * HW;
    float v[9];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        int yy = y + ky - 1, xx = x + kx - 1;
        v[ky * 3 + kx] = (yy >= 0 && yy < H && xx >= 0 && xx < H) ? ic[yy * H + xx] : 0.f;
      }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int co = 4 * g + j;
      if (co >= cout) break;
      const __nv_bfloat16* w = W + ((size_t)co * cin + ci) * 9;
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[j] = fmaf(__bfloat162float(w[k]), v[k], acc[j]);
    }
  }
  float* ob = out + (size_t)b * out_ctot * HW;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int co = 4 * g + j;
    if (co >= cout) break;
    ob[(size_t)co * HW + pix] = relu ? fmaxf(acc[j], 0.f) : acc[j];
  }
}

// din[b][ci][y][x] = sum_co,ky,kx W[co][ci][ky][kx] dout[b][co][y-ky+1][x-kx+1]
__global__ void k_conv_bwd_data(const float* __restrict__ dout, int dout_ctot, int cout,
                                const __nv_bfloat16* __restrict__ W, float* __restrict__ din,
                                int din_ctot, int cin, int B, int H, int accumulate) {
  const int HW = H * H;
  const int cg = (cin + 3) / 4;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  long long total = (long long)B * cg * HW;
  if (t >= total) return;
  int pix = (int)(t % HW);
  int g = (int)((t / HW) % cg);
  int b = (int)(t / ((long long)HW * cg));
  int y = pix / H, x = pix % H;
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  const float* db = dout + (size_t)b * dout_ctot * HW;
  for (int co = 0; co < cout; ++co) {
    const float* dc = db + (size_t)co * HW;
    float v[9];
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        int yy = y - ky + 1, xx = x - kx + 1;
        v[ky * 3 + kx] = (yy >= 0 && yy < H && xx >= 0 && xx < H) ? dc[yy * H + xx] : 0.f;
      }
#pragma unroll
    for (int j = 0; j < 4; ++j) {
      int ci = 4 * g + j;
      if (ci >= cin) break;
      const __nv_bfloat16* w = W + ((size_t)co * cin + ci) * 9;
#pragma unroll
      for (int k = 0; k < 9; ++k) acc[j] = fmaf(__bfloat162float(w[k]), v[k], acc[j]);
    }
  }
  float* ob = din + (size_t)b * din_ctot * HW;
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    int ci = 4 * g + j;
    if (ci >= cin) break;
    size_t o = (size_t)ci * HW + pix;
    ob[o] = accumulate ? ob[o] + acc[j] : acc[j];
  }
}

// dW[co][ci][k] = sum_b,y,x dout[b][co][y][x] in[b][ci][y+ky-1][x+kx-1]; one
// block per (co, ci); db[co] from the blocks with ci == 0. Fixed-order
// reduction (deterministic).
__global__ void k_conv_bwd_w(const float* __restrict__ in, int in_ctot, int cin,
                             const float* __restrict__ dout, int dout_ctot, int cout, int B, int H,
                             float* __restrict__ dW, float* __restrict__ dbias) {
  const int co = blockIdx.x / cin, ci = blockIdx.x % cin;
  const int HW = H * H;
  float acc[10] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};
  for (long long t = threadIdx.x; t < (long long)B * HW; t += blockDim.x) {
    int b = (int)(t / HW), pix = (int)(t % HW);
    int y = pix / H, x = pix % H;
    float g = dout[((size_t)b * dout_ctot + co) * HW + pix];
    const float* ic = in + ((size_t)b * in_ctot + ci) * HW;
#pragma unroll
    for (int ky = 0; ky < 3; ++ky)
#pragma unroll
      for (int kx = 0; kx < 3; ++kx) {
        int yy = y + ky - 1, xx = x + kx - 1;
        float v = (yy >= 0 && yy < H && xx >= 0 && xx < H) ? ic[yy * H + xx] : 0.f;
        acc[ky * 3 + kx] = fmaf(g, v, acc[ky * 3 + kx]);
      }
    acc[9] += g;
  }
  __shared__ float red[10][32];
  const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
#pragma unroll
  for (int k = 0; k < 10; ++k) {
    float v = acc[k];
    for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
    if (lane == 0) red[k][w] = v;
  }
  __syncthreads();
  if (threadIdx.x < 10) {
    float s = 0.f;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[threadIdx.x][i];
    if (threadIdx.x < 9) dW[((size_t)co * cin + ci) * 9 + threadIdx.x] = s;
    else if (ci == 0) dbias[co] = s;
  }
}

__global__ void k_relu_bwd(const float* __restrict__ act, int act_ctot, float* __restrict__ d,
                           int d_ctot, int c, int B, int HW) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * c * HW) return;
  int pix = (int)(t % HW), ch = (int)((t / HW) % c), b = (int)(t / ((long long)HW * c));
  if (act[((size_t)b * act_ctot + ch) * HW + pix] <= 0.f) d[((size_t)b * d_ctot + ch) * HW + pix] = 0.f;
}

// 2x2 average pool (H -> H/2)
__global__ void k_pool_fwd(const float* __restrict__ in, int in_ctot, float* __restrict__ out,
                           int out_ctot, int c, int B, int H) {
  const int h = H / 2;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * c * h * h) return;
  int pix = (int)(t % (h * h)), ch = (int)((t / (h * h)) % c), b = (int)(t / ((long long)h * h * c));
  int y = pix / h, x = pix % h;
  const float* i = in + ((size_t)b * in_ctot + ch) * H * H;
  out[((size_t)b * out_ctot + ch) * h * h + pix] =
      0.25f * (i[(2 * y) * H + 2 * x] + i[(2 * y) * H + 2 * x + 1] + i[(2 * y + 1) * H + 2 * x] +
               i[(2 * y + 1) * H + 2 * x + 1]);
}

// gradient of the pool, accumulated into din (H x H)
__global__ void k_pool_bwd(const float* __restrict__ dout, int dout_ctot, float* __restrict__ din,
                           int din_ctot, int c, int B, int H) {
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * c * H * H) return;
  int pix = (int)(t % (H * H)), ch = (int)((t / (H * H)) % c), b = (int)(t / ((long long)H * H * c));
  int y = pix / H, x = pix % H, h = H / 2;
  din[((size_t)b * din_ctot + ch) * H * H + pix] +=
      0.25f * dout[((size_t)b * dout_ctot + ch) * h * h + (y / 2) * h + x / 2];
}

// nearest 2x upsample (h -> 2h)
__global__ void k_up_fwd(const float* __restrict__ in, int in_ctot, float* __restrict__ out,
                         int out_ctot, int c, int B, int h) {
  const int H = 2 * h;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * c * H * H) return;
  int pix = (int)(t % (H * H)), ch = (int)((t / (H * H)) % c), b = (int)(t / ((long long)H * H * c));
  int y = pix / H, x = pix % H;
  out[((size_t)b * out_ctot + ch) * H * H + pix] = in[((size_t)b * in_ctot + ch) * h * h + (y / 2) * h + x / 2];
}

__global__ void k_up_bwd(const float* __restrict__ dout, int dout_ctot, float* __restrict__ din,
                         int din_ctot, int c, int B, int h) {
  const int H = 2 * h;
  long long t = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (t >= (long long)B * c * h * h) return;
  int pix = (int)(t % (h * h)), ch = (int)((t / (h * h)) % c), b = (int)(t / ((long long)h * h * c));
  int y = pix / h, x = pix % h;
  const float* d = dout + ((size_t)b * dout_ctot + ch) * H * H;
  din[((size_t)b * din_ctot + ch) * h * h + pix] =
      d[(2 * y) * H + 2 * x] + d[(2 * y) * H + 2 * x + 1] + d[(2 * y + 1) * H + 2 * x] +
      d[(2 * y + 1) * H + 2 * x + 1];
}

// MSE: loss = mean (y - t)^2 ; grad = 2 (y - t) / count. Partial sums per block.
__global__ void k_mse(const float* __restrict__ y, const float* __restrict__ t, long long count,
                      float* __restrict__ grad, double* __restrict__ partial) {
  double acc = 0.0;
  for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < count;
       i += (long long)gridDim.x * blockDim.x) {
    float d = y[i] - t[i];
    grad[i] = 2.f * d / (float)count;
    acc += (double)d * d;
  }
  __shared__ double red[32];
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double s = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) s += red[i];
    partial[blockIdx.x] = s;
  }
}

__global__ void k_adam(float* __restrict__ p, const float* __restrict__ g, float* __restrict__ m,
                       float* __restrict__ v, __nv_bfloat16* __restrict__ pb, int n_w, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= n) return;
  float gi = g[i];
  float mi = b1 * m[i] + (1.f - b1) * gi;
  float vi = b2 * v[i] + (1.f - b2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  float pi = p[i] - lr * (mi / c1) / (sqrtf(vi / c2) + eps);
  p[i] = pi;
  if (i < n_w) pb[i] = __float2bfloat16_rn(pi);
}

__global__ void k_to_bf16(const float* __restrict__ p, __nv_bfloat16* __restrict__ pb, int n) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < n) pb[i] = __float2bfloat16_rn(p[i]);
}

// ---- warm-start features / targets / apply (maps [count][n][n], R | n)
__global__ void k_warm_features(const float* __restrict__ th1, const float* __restrict__ pl,
                                const float* __restrict__ s, int n, int R, float* __restrict__ x) {
  const int b = blockIdx.x;
  const size_t nn = (size_t)n * n;
  const float* plb = pl + b * nn;
  double acc = 0.0;
  for (size_t i = threadIdx.x; i < nn; i += blockDim.x) acc += plb[i];
  __shared__ double red[32];
  __shared__ float mean_s;
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = acc;
  __syncthreads();
  if (threadIdx.x == 0) {
    double t = 0.0;
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) t += red[i];
    mean_s = (float)(t / (double)nn);
  }
  __syncthreads();
  const float mean = mean_s;
  const int f = n / R;
  const float inv = 1.f / (float)(f * f);
  for (int o = threadIdx.x; o < R * R; o += blockDim.x) {
    int Y = o / R, X = o % R;
    float a = 0.f, c = 0.f, e = 0.f;
    for (int dy = 0; dy < f; ++dy)
      for (int dx = 0; dx < f; ++dx) {
        size_t idx = b * nn + (size_t)(Y * f + dy) * n + X * f + dx;
        a += th1[idx];
        c += pl[idx];
        e += s ? s[idx] : 1.f;
      }
    float* xb = x + (size_t)b * 3 * R * R;
    xb[o] = a * inv / 100.f;
    xb[R * R + o] = 10.f * (c * inv / mean - 1.f);
    xb[2 * R * R + o] = 30.f * (e * inv - 1.f);
  }
}

__global__ void k_warm_target(const float* __restrict__ ths, const float* __restrict__ th1, int n,
                              int R, int count, float* __restrict__ t) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)count * R * R) return;
  int b = (int)(i / (R * R)), o = (int)(i % (R * R));
  int Y = o / R, X = o % R, f = n / R;
  float a = 0.f;
  for (int dy = 0; dy < f; ++dy)
    for (int dx = 0; dx < f; ++dx) {
      size_t idx = (size_t)b * n * n + (size_t)(Y * f + dy) * n + X * f + dx;
      a += ths[idx] - th1[idx];
    }
  t[i] = a / (float)(f * f) / 10.f;
}

// theta_init = theta_1 + 10 * bilinear(y) (cell-centred, edge clamped)
__global__ void k_warm_apply(const float* __restrict__ th1, const float* __restrict__ y, int n,
                             int R, int count, float* __restrict__ out) {
  long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= (long long)count * n * n) return;
  int b = (int)(i / ((long long)n * n));
  int pix = (int)(i % ((long long)n * n));
  int yy = pix / n, xx = pix % n;
  float sc = (float)R / (float)n;
  float fy = fminf(fmaxf((yy + 0.5f) * sc - 0.5f, 0.f), (float)(R - 1));
  float fx = fminf(fmaxf((xx + 0.5f) * sc - 0.5f, 0.f), (float)(R - 1));
  int y0 = (int)fy, x0 = (int)fx;
  int y1 = min(y0 + 1, R - 1), x1 = min(x0 + 1, R - 1);
  float wy = fy - y0, wx = fx - x0;
  const float* yb = y + (size_t)b * R * R;
  float v = (1.f - wy) * ((1.f - wx) * yb[y0 * R + x0] + wx * yb[y0 * R + x1]) +
            wy * ((1.f - wx) * yb[y1 * R + x0] + wx * yb[y1 * R + x1]);
  out[i] = th1[i] + 10.f * v;
}

inline unsigned blocks(long long n, int t) { return (unsigned)((n + t - 1) / t); }

uint64_t splitmix(uint64_t& s) {
  uint64_t z = (s += 0x9E3779B97F4A7C15ull);
  z = (z ^ (z >> 30)) * 0xBF58476D1CE4E5B9ull;
  z = (z ^ (z >> 27)) * 0x94D049BB133111EBull;
  return z ^ (z >> 31);
}

}  // namespace

// ---------------------------------------------------------------- model
struct vs_model_t {
  int C, R;
  int cin[kLayers], cout[kLayers], res[kLayers], relu[kLayers];
  size_t woff[kLayers], boff[kLayers];
  size_t n_w, n_params;        // weights first, then biases
  float* p = nullptr;          // master FP32 params
  float* g = nullptr;          // gradients
  float* m = nullptr;
  float* v = nullptr;
  __nv_bfloat16* pb = nullptr; // BF16 copy of the weights
  long long step = 0;
  // activations for a max batch
  int maxB = 0;
  float *x = nullptr, *a1 = nullptr, *c2 = nullptr, *p1 = nullptr, *a3 = nullptr, *c1 = nullptr,
        *p2 = nullptr, *a5 = nullptr, *a6 = nullptr, *a7 = nullptr, *y = nullptr;
  float *dy = nullptr, *da7 = nullptr, *dc2 = nullptr, *da6 = nullptr, *dc1 = nullptr,
        *da5 = nullptr, *dp2 = nullptr, *da3 = nullptr, *dp1 = nullptr, *da1 = nullptr;
  double* partial = nullptr;
};

namespace {

void free_acts(vs_model_t* m) {
  float** a[] = {&m->x, &m->a1, &m->c2, &m->p1, &m->a3, &m->c1, &m->p2, &m->a5, &m->a6, &m->a7,
                 &m->y, &m->dy, &m->da7, &m->dc2, &m->da6, &m->dc1, &m->da5, &m->dp2, &m->da3,
                 &m->dp1, &m->da1};
  for (auto pp : a) {
    cudaFree(*pp);
    *pp = nullptr;
  }
  cudaFree(m->partial);
  m->partial = nullptr;
  m->maxB = 0;
}

int ensure_acts(vs_model_t* m, int B) {
  if (B <= m->maxB) return VS_OK;
  free_acts(m);
  const size_t R2 = (size_t)m->R * m->R, h2 = R2 / 4, q2 = R2 / 16;
  const int C = m->C;
  struct Buf { float** p; size_t n; } bufs[] = {
      {&m->x, 3 * R2}, {&m->a1, C * R2}, {&m->c2, 2 * C * R2}, {&m->p1, C * h2},
      {&m->a3, 2 * C * h2}, {&m->c1, 4 * C * h2}, {&m->p2, 2 * C * q2}, {&m->a5, 2 * C * q2},
      {&m->a6, C * h2}, {&m->a7, C * R2}, {&m->y, R2}, {&m->dy, R2}, {&m->da7, C * R2},
      {&m->dc2, 2 * C * R2}, {&m->da6, C * h2}, {&m->dc1, 4 * C * h2}, {&m->da5, 2 * C * q2},
      {&m->dp2, 2 * C * q2}, {&m->da3, 2 * C * h2}, {&m->dp1, C * h2}, {&m->da1, C * R2}};
  for (auto& b : bufs) VS_CUDA_TRY(cudaMalloc(b.p, sizeof(float) * b.n * B));
  VS_CUDA_TRY(cudaMalloc(&m->partial, sizeof(double) * 1024));
  m->maxB = B;
  return VS_OK;
}

void conv_fwd(vs_model_t* m, int l, TView in, TView out, int B, cudaStream_t s, bool tc = false) {
  int H = m->res[l];
  if (tc) {
    // tensor cores where the layer's shape fits (inference); else the SIMT kernel
    const int rc = vs_conv_tc(in.p, in.ctot, m->cin[l], m->pb + m->woff[l], m->p + m->boff[l], out.p,
                              out.ctot, m->cout[l], B, H, m->relu[l], s);
    if (rc != -1) return;
  }
  long long total = (long long)B * ((m->cout[l] + 3) / 4) * H * H;
  k_conv_fwd<<<blocks(total, 256), 256, 0, s>>>(in.p, in.ctot, m->cin[l], m->pb + m->woff[l],
                                                m->p + m->boff[l], out.p, out.ctot, m->cout[l], B,
                                                H, m->relu[l]);
}

void conv_bwd(vs_model_t* m, int l, TView in, TView dout, TView din, int B, bool need_din,
              bool accumulate, cudaStream_t s) {
  int H = m->res[l];
  k_conv_bwd_w<<<m->cout[l] * m->cin[l], 256, 0, s>>>(in.p, in.ctot, m->cin[l], dout.p, dout.ctot,
                                                      m->cout[l], B, H, m->g + m->woff[l],
                                                      m->g + m->boff[l]);
  if (need_din) {
    long long total = (long long)B * ((m->cin[l] + 3) / 4) * H * H;
    k_conv_bwd_data<<<blocks(total, 256), 256, 0, s>>>(dout.p, dout.ctot, m->cout[l],
                                                       m->pb + m->woff[l], din.p, din.ctot,
                                                       m->cin[l], B, H, accumulate ? 1 : 0);
  }
}

void relu_bwd(TView act, TView d, int c, int B, int H, cudaStream_t s) {
  long long total = (long long)B * c * H * H;
  k_relu_bwd<<<blocks(total, 256), 256, 0, s>>>(act.p, act.ctot, d.p, d.ctot, c, B, H * H);
}

// forward of a batch already in m->x; tc: the convolutions on the tensor
// cores (BF16 activations, inference) where their shapes fit
void forward(vs_model_t* m, int B, cudaStream_t s, bool tc = false) {
  const int C = m->C, R = m->R, h = R / 2, q = R / 4;
  const size_t R2 = (size_t)R * R, h2 = (size_t)h * h;
  conv_fwd(m, 0, {m->x, 3}, {m->a1, C}, B, s, tc);
  conv_fwd(m, 1, {m->a1, C}, {m->c2 + C * R2, 2 * C}, B, s, tc);            // s1 into c2[C:2C)
  k_pool_fwd<<<blocks((long long)B * C * h2, 256), 256, 0, s>>>(m->c2 + C * R2, 2 * C, m->p1, C, C, B, R);
  conv_fwd(m, 2, {m->p1, C}, {m->a3, 2 * C}, B, s, tc);
  conv_fwd(m, 3, {m->a3, 2 * C}, {m->c1 + 2 * C * h2, 4 * C}, B, s, tc);    // s2 into c1[2C:4C)
  k_pool_fwd<<<blocks((long long)B * 2 * C * q * q, 256), 256, 0, s>>>(m->c1 + 2 * C * h2, 4 * C, m->p2,
                                                                     2 * C, 2 * C, B, h);
  conv_fwd(m, 4, {m->p2, 2 * C}, {m->a5, 2 * C}, B, s, tc);
  k_up_fwd<<<blocks((long long)B * 2 * C * h2, 256), 256, 0, s>>>(m->a5, 2 * C, m->c1, 4 * C, 2 * C, B, q);
  conv_fwd(m, 5, {m->c1, 4 * C}, {m->a6, C}, B, s, tc);
  k_up_fwd<<<blocks((long long)B * C * R2, 256), 256, 0, s>>>(m->a6, C, m->c2, 2 * C, C, B, h);
  conv_fwd(m, 6, {m->c2, 2 * C}, {m->a7, C}, B, s, tc);
  conv_fwd(m, 7, {m->a7, C}, {m->y, 1}, B, s, tc);
}

// backward from m->dy; fills m->g
void backward(vs_model_t* m, int B, cudaStream_t s) {
  const int C = m->C, R = m->R, h = R / 2, q = R / 4;
  const size_t R2 = (size_t)R * R, h2 = (size_t)h * h;
  conv_bwd(m, 7, {m->a7, C}, {m->dy, 1}, {m->da7, C}, B, true, false, s);
  relu_bwd({m->a7, C}, {m->da7, C}, C, B, R, s);
  conv_bwd(m, 6, {m->c2, 2 * C}, {m->da7, C}, {m->dc2, 2 * C}, B, true, false, s);
  // dc2[0:C) -> up -> da6 ; dc2[C:2C) is d(s1), completed below by the pool path
  k_up_bwd<<<blocks((long long)B * C * h2, 256), 256, 0, s>>>(m->dc2, 2 * C, m->da6, C, C, B, h);
  relu_bwd({m->a6, C}, {m->da6, C}, C, B, h, s);
  conv_bwd(m, 5, {m->c1, 4 * C}, {m->da6, C}, {m->dc1, 4 * C}, B, true, false, s);
  k_up_bwd<<<blocks((long long)B * 2 * C * q * q, 256), 256, 0, s>>>(m->dc1, 4 * C, m->da5, 2 * C, 2 * C, B, q);
  relu_bwd({m->a5, 2 * C}, {m->da5, 2 * C}, 2 * C, B, q, s);
  conv_bwd(m, 4, {m->p2, 2 * C}, {m->da5, 2 * C}, {m->dp2, 2 * C}, B, true, false, s);
  k_pool_bwd<<<blocks((long long)B * 2 * C * h2, 256), 256, 0, s>>>(m->dp2, 2 * C, m->dc1 + 2 * C * h2, 4 * C,
                                                                 2 * C, B, h);
  relu_bwd({m->c1 + 2 * C * h2, 4 * C}, {m->dc1 + 2 * C * h2, 4 * C}, 2 * C, B, h, s);
  conv_bwd(m, 3, {m->a3, 2 * C}, {m->dc1 + 2 * C * h2, 4 * C}, {m->da3, 2 * C}, B, true, false, s);
  relu_bwd({m->a3, 2 * C}, {m->da3, 2 * C}, 2 * C, B, h, s);
  conv_bwd(m, 2, {m->p1, C}, {m->da3, 2 * C}, {m->dp1, C}, B, true, false, s);
  k_pool_bwd<<<blocks((long long)B * C * R2, 256), 256, 0, s>>>(m->dp1, C, m->dc2 + C * R2, 2 * C, C, B, R);
  relu_bwd({m->c2 + C * R2, 2 * C}, {m->dc2 + C * R2, 2 * C}, C, B, R, s);
  conv_bwd(m, 1, {m->a1, C}, {m->dc2 + C * R2, 2 * C}, {m->da1, C}, B, true, false, s);
  relu_bwd({m->a1, C}, {m->da1, C}, C, B, R, s);
  conv_bwd(m, 0, {m->x, 3}, {m->da1, C}, {nullptr, 0}, B, false, false, s);
}

int loss_grad(vs_model_t* m, const float* x, const float* t, int B, double* loss, cudaStream_t s) {
  int rc = ensure_acts(m, B);
  if (rc) return rc;
  const size_t R2 = (size_t)m->R * m->R;
  VS_CUDA_TRY(cudaMemcpyAsync(m->x, x, sizeof(float) * 3 * R2 * B, cudaMemcpyDeviceToDevice, s));
  forward(m, B, s);
  long long count = (long long)B * R2;
  int nb = (int)std::min<long long>(1024, blocks(count, 256));
  k_mse<<<nb, 256, 0, s>>>(m->y, t, count, m->dy, m->partial);
  backward(m, B, s);
  VS_CUDA_TRY(cudaGetLastError());
  if (loss) {
    std::vector<double> part(nb);
    VS_CUDA_TRY(cudaMemcpyAsync(part.data(), m->partial, sizeof(double) * nb, cudaMemcpyDeviceToHost, s));
    VS_CUDA_TRY(cudaStreamSynchronize(s));
    double tot = 0.0;
    for (double v : part) tot += v;
    *loss = tot / (double)count;
  }
  return VS_OK;
}

}  // namespace

extern "C" int vs_model_create(int base_channels, int resolution, unsigned long long seed,
                               vs_model* out) {
  if (!out) return vs_set_error(VS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (base_channels < 1 || base_channels > 64)
    return vs_set_error(VS_ERR_INVALID_ARG, "base_channels %d outside [1, 64]", base_channels);
  if (resolution < 8 || resolution > 256 || (resolution % 4))
    return vs_set_error(VS_ERR_INVALID_ARG, "resolution %d must be a multiple of 4 in [8, 256]",
                        resolution);
  vs_model_t* m = new vs_model_t();
  const int C = base_channels, R = resolution;
  m->C = C;
  m->R = R;
  const int ci[kLayers] = {3, C, C, 2 * C, 2 * C, 4 * C, 2 * C, C};
  const int co[kLayers] = {C, C, 2 * C, 2 * C, 2 * C, C, C, 1};
  const int rs[kLayers] = {R, R, R / 2, R / 2, R / 4, R / 2, R, R};
  size_t off = 0;
  for (int l = 0; l < kLayers; ++l) {
    m->cin[l] = ci[l];
    m->cout[l] = co[l];
    m->res[l] = rs[l];
    m->relu[l] = l < kLayers - 1;
    m->woff[l] = off;
    off += (size_t)co[l] * ci[l] * 9;
  }
  m->n_w = off;
  for (int l = 0; l < kLayers; ++l) {
    m->boff[l] = off;
    off += co[l];
  }
  m->n_params = off;
  // He-uniform weights, zero biases, from a splitmix64 stream
  std::vector<float> h(m->n_params, 0.f);
  uint64_t st = seed;
  for (int l = 0; l < kLayers; ++l) {
    float lim = sqrtf(6.f / (9.f * ci[l])) * (l == kLayers - 1 ? 0.1f : 1.f);
    for (size_t i = 0; i < (size_t)co[l] * ci[l] * 9; ++i) {
      double u = (double)(splitmix(st) >> 11) * (1.0 / 9007199254740992.0);
      h[m->woff[l] + i] = (float)((2.0 * u - 1.0) * lim);
    }
  }
  auto fail = [&](cudaError_t e) {
    vs_free_model(m);
    return vs_set_error(e == cudaErrorMemoryAllocation ? VS_ERR_OOM : VS_ERR_CUDA, "model: %s",
                        cudaGetErrorString(e));
  };
  cudaError_t e;
  if ((e = cudaMalloc(&m->p, sizeof(float) * m->n_params))) return fail(e);
  if ((e = cudaMalloc(&m->g, sizeof(float) * m->n_params))) return fail(e);
  if ((e = cudaMalloc(&m->m, sizeof(float) * m->n_params))) return fail(e);
  if ((e = cudaMalloc(&m->v, sizeof(float) * m->n_params))) return fail(e);
  if ((e = cudaMalloc(&m->pb, sizeof(__nv_bfloat16) * m->n_w))) return fail(e);
  if ((e = cudaMemcpy(m->p, h.data(), sizeof(float) * m->n_params, cudaMemcpyHostToDevice))) return fail(e);
  if ((e = cudaMemset(m->m, 0, sizeof(float) * m->n_params))) return fail(e);
  if ((e = cudaMemset(m->v, 0, sizeof(float) * m->n_params))) return fail(e);
  k_to_bf16<<<blocks((long long)m->n_w, 256), 256>>>(m->p, m->pb, (int)m->n_w);
  if ((e = cudaDeviceSynchronize())) return fail(e);
  *out = m;
  return VS_OK;
}

extern "C" void vs_free_model(vs_model m) {
  if (!m) return;
  free_acts(m);
  cudaFree(m->p);
  cudaFree(m->g);
  cudaFree(m->m);
  cudaFree(m->v);
  cudaFree(m->pb);
  delete m;
}

extern "C" long long vs_model_nparams(vs_model m) { return m ? (long long)m->n_params : -1; }

extern "C" int vs_model_get_params(vs_model m, float* host) {
  if (!m || !host) return vs_set_error(VS_ERR_INVALID_ARG, "NULL model or output");
  VS_CUDA_TRY(cudaMemcpy(host, m->p, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
  return VS_OK;
}

extern "C" int vs_model_set_params(vs_model m, const float* host) {
  if (!m || !host) return vs_set_error(VS_ERR_INVALID_ARG, "NULL model or input");
  VS_CUDA_TRY(cudaMemcpy(m->p, host, sizeof(float) * m->n_params, cudaMemcpyHostToDevice));
  k_to_bf16<<<blocks((long long)m->n_w, 256), 256>>>(m->p, m->pb, (int)m->n_w);
  VS_CUDA_TRY(cudaMemset(m->m, 0, sizeof(float) * m->n_params));
  VS_CUDA_TRY(cudaMemset(m->v, 0, sizeof(float) * m->n_params));
  m->step = 0;
  VS_CUDA_TRY(cudaDeviceSynchronize());
  return VS_OK;
}

namespace {
int model_forward(vs_model m, const float* x, float* y, int batch, void* stream, bool tc) {
  if (!m || !x || !y || batch < 1) return vs_set_error(VS_ERR_INVALID_ARG, "bad model forward arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t R2 = (size_t)m->R * m->R;
  const int chunk = 256;
  int rc = ensure_acts(m, std::min(batch, chunk));
  if (rc) return rc;
  for (int b0 = 0; b0 < batch; b0 += chunk) {
    int B = std::min(chunk, batch - b0);
    VS_CUDA_TRY(cudaMemcpyAsync(m->x, x + (size_t)b0 * 3 * R2, sizeof(float) * 3 * R2 * B,
                                cudaMemcpyDeviceToDevice, s));
    forward(m, B, s, tc);
    VS_CUDA_TRY(cudaMemcpyAsync(y + (size_t)b0 * R2, m->y, sizeof(float) * R2 * B,
                                cudaMemcpyDeviceToDevice, s));
  }
  VS_CUDA_TRY(cudaGetLastError());
  return VS_OK;
}
}  // namespace

extern "C" int vs_model_forward(vs_model m, const float* x, float* y, int batch, void* stream) {
  return model_forward(m, x, y, batch, stream, false);
}

extern "C" int vs_model_forward_tc(vs_model m, const float* x, float* y, int batch, void* stream) {
  return model_forward(m, x, y, batch, stream, true);
}

extern "C" int vs_model_loss_grad(vs_model m, const float* x, const float* t, int batch,
                                  double* loss_host, float* grad_host, void* stream) {
  if (!m || !x || !t || batch < 1) return vs_set_error(VS_ERR_INVALID_ARG, "bad loss_grad arguments");
  cudaStream_t s = (cudaStream_t)stream;
  int rc = loss_grad(m, x, t, batch, loss_host, s);
  if (rc) return rc;
  if (grad_host) {
    VS_CUDA_TRY(cudaMemcpyAsync(grad_host, m->g, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost, s));
    VS_CUDA_TRY(cudaStreamSynchronize(s));
  }
  return VS_OK;
}

extern "C" int vs_model_train(vs_model m, const float* x, const float* t, int n_samples, int epochs,
                              int batch, float lr, unsigned long long seed, double* loss_host,
                              void* stream) {
  if (!m || !x || !t || n_samples < batch || batch < 1 || epochs < 1 || !(lr > 0.f))
    return vs_set_error(VS_ERR_INVALID_ARG, "bad training arguments");
  cudaStream_t s = (cudaStream_t)stream;
  const size_t R2 = (size_t)m->R * m->R;
  int rc = ensure_acts(m, batch);
  if (rc) return rc;
  float* tb = nullptr;
  VS_CUDA_TRY(cudaMallocAsync(&tb, sizeof(float) * R2 * batch, s));
  std::vector<int> order(n_samples);
  for (int i = 0; i < n_samples; ++i) order[i] = i;
  uint64_t st = seed;
  double last = 0.0;
  const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
  for (int ep = 0; ep < epochs; ++ep) {
    for (int i = n_samples - 1; i > 0; --i) {     // Fisher-Yates
      int j = (int)(splitmix(st) % (uint64_t)(i + 1));
      std::swap(order[i], order[j]);
    }
    double ep_loss = 0.0;
    int nb = 0;
    for (int b0 = 0; b0 + batch <= n_samples; b0 += batch) {
      for (int k = 0; k < batch; ++k) {
        int idx = order[b0 + k];
        VS_CUDA_TRY(cudaMemcpyAsync(m->x + (size_t)k * 3 * R2, x + (size_t)idx * 3 * R2,
                                    sizeof(float) * 3 * R2, cudaMemcpyDeviceToDevice, s));
        VS_CUDA_TRY(cudaMemcpyAsync(tb + (size_t)k * R2, t + (size_t)idx * R2, sizeof(float) * R2,
                                    cudaMemcpyDeviceToDevice, s));
      }
      forward(m, batch, s);
      long long count = (long long)batch * R2;
      int nbk = (int)std::min<long long>(1024, blocks(count, 256));
      k_mse<<<nbk, 256, 0, s>>>(m->y, tb, count, m->dy, m->partial);
      backward(m, batch, s);
      m->step++;
      float c1 = 1.f - powf(b1, (float)m->step), c2 = 1.f - powf(b2, (float)m->step);
      k_adam<<<blocks((long long)m->n_params, 256), 256, 0, s>>>(m->p, m->g, m->m, m->v, m->pb,
                                                                (int)m->n_w, (int)m->n_params, lr,
                                                                b1, b2, eps, c1, c2);
      if (b0 + 2 * batch > n_samples) {            // loss of the last batch of the epoch
        std::vector<double> part(nbk);
        VS_CUDA_TRY(cudaMemcpyAsync(part.data(), m->partial, sizeof(double) * nbk,
                                    cudaMemcpyDeviceToHost, s));
        VS_CUDA_TRY(cudaStreamSynchronize(s));
        double tot = 0.0;
        for (double v : part) tot += v;
        ep_loss = tot / (double)count;
      }
      ++nb;
    }
    last = ep_loss;
  }
  VS_CUDA_TRY(cudaGetLastError());
  VS_CUDA_TRY(cudaFreeAsync(tb, s));
  VS_CUDA_TRY(cudaStreamSynchronize(s));
  if (loss_host) *loss_host = last;
  return VS_OK;
}

extern "C" int vs_model_save(vs_model m, const char* path) {
  if (!m || !path) return vs_set_error(VS_ERR_INVALID_ARG, "NULL model or path");
  std::vector<float> h(m->n_params);
  VS_CUDA_TRY(cudaMemcpy(h.data(), m->p, sizeof(float) * m->n_params, cudaMemcpyDeviceToHost));
  FILE* f = fopen(path, "wb");
  if (!f) return vs_set_error(VS_ERR_INVALID_ARG, "cannot open %s", path);
  const char magic[8] = {'V', 'S', 'C', 'N', 'N', '0', '0', '1'};
  int hdr[2] = {m->C, m->R};
  long long np = (long long)m->n_params;
  bool ok = fwrite(magic, 1, 8, f) == 8 && fwrite(hdr, sizeof(int), 2, f) == 2 &&
            fwrite(&np, sizeof(np), 1, f) == 1 && fwrite(h.data(), sizeof(float), h.size(), f) == h.size();
  fclose(f);
  return ok ? VS_OK : vs_set_error(VS_ERR_INVALID_ARG, "write failed: %s", path);
}

extern "C" int vs_model_load(const char* path, vs_model* out) {
  if (!path || !out) return vs_set_error(VS_ERR_INVALID_ARG, "NULL path or output");
  *out = nullptr;
  FILE* f = fopen(path, "rb");
  if (!f) return vs_set_error(VS_ERR_INVALID_ARG, "cannot open %s", path);
  char magic[8];
  int hdr[2];
  long long np = 0;
  bool ok = fread(magic, 1, 8, f) == 8 && memcmp(magic, "VSCNN001", 8) == 0 &&
            fread(hdr, sizeof(int), 2, f) == 2 && fread(&np, sizeof(np), 1, f) == 1;
  if (!ok) {
    fclose(f);
    return vs_set_error(VS_ERR_INVALID_ARG, "%s is not a model checkpoint", path);
  }
  vs_model m = nullptr;
  int rc = vs_model_create(hdr[0], hdr[1], 0, &m);
  if (rc) {
    fclose(f);
    return rc;
  }
  if ((long long)m->n_params != np) {
    fclose(f);
    vs_free_model(m);
    return vs_set_error(VS_ERR_INVALID_ARG, "checkpoint parameter count mismatch");
  }
  std::vector<float> h(np);
  ok = fread(h.data(), sizeof(float), h.size(), f) == h.size();
  fclose(f);
  if (!ok) {
    vs_free_model(m);
    return vs_set_error(VS_ERR_INVALID_ARG, "truncated checkpoint %s", path);
  }
  rc = vs_model_set_params(m, h.data());
  if (rc) {
    vs_free_model(m);
    return rc;
  }
  *out = m;
  return VS_OK;
}

extern "C" int vs_warm_features(const float* theta1, const float* p_leak0, const float* s_kappa,
                                int count, int n, int resolution, float* x_out, void* stream) {
  if (!theta1 || !p_leak0 || !x_out || count < 1 || resolution < 4 || n % resolution)
    return vs_set_error(VS_ERR_INVALID_ARG, "bad warm-feature arguments");
  k_warm_features<<<count, 256, 0, (cudaStream_t)stream>>>(theta1, p_leak0, s_kappa, n, resolution, x_out);
  VS_CUDA_TRY(cudaGetLastError());
  return VS_OK;
}

extern "C" int vs_warm_target(const float* theta_star, const float* theta1, int count, int n,
                              int resolution, float* t_out, void* stream) {
  if (!theta_star || !theta1 || !t_out || count < 1 || resolution < 4 || n % resolution)
    return vs_set_error(VS_ERR_INVALID_ARG, "bad warm-target arguments");
  long long total = (long long)count * resolution * resolution;
  k_warm_target<<<blocks(total, 256), 256, 0, (cudaStream_t)stream>>>(theta_star, theta1, n,
                                                                      resolution, count, t_out);
  VS_CUDA_TRY(cudaGetLastError());
  return VS_OK;
}

extern "C" int vs_warm_apply(const float* theta1, const float* y, int count, int n, int resolution,
                             float* theta_init, void* stream) {
  if (!theta1 || !y || !theta_init || count < 1 || resolution < 4 || n % resolution)
    return vs_set_error(VS_ERR_INVALID_ARG, "bad warm-apply arguments");
  long long total = (long long)count * n * n;
  k_warm_apply<<<blocks(total, 256), 256, 0, (cudaStream_t)stream>>>(theta1, y, n, resolution,
                                                                     count, theta_init);
  VS_CUDA_TRY(cudaGetLastError());
  return VS_OK;
}

extern "C" int vs_model_shape(vs_model m, int* base_channels, int* resolution) {
  if (!m || !base_channels || !resolution) return vs_set_error(VS_ERR_INVALID_ARG, "NULL model or output");
  *base_channels = m->C;
  *resolution = m->R;
  return VS_OK;
}

// ---------------------------------------------------------------------------
// Warm-started batched solve: first iterate -> network -> warm solve, with a
// cold re-solve of the maps the warm start did not bring to convergence.
// ---------------------------------------------------------------------------

struct vs_warm_plan_t {
  vs_kernel k = nullptr;
  vs_model model = nullptr;
  int count = 0, n = 0, R = 0;
  const float *pd = nullptr, *pl = nullptr, *sk = nullptr;
  float *theta = nullptr, *theta1 = nullptr, *theta_init = nullptr;
  float *x = nullptr, *y = nullptr;      // network input / output, owned
  vs_plan first = nullptr, warm = nullptr;
  vs_solve_params params;
};

namespace {

// Outcomes that belong to single maps (the rest fail the whole launch).
bool per_map_status(int rc) {
  return rc == VS_OK || rc == VS_ERR_NO_CONVERGENCE || rc == VS_ERR_RUNAWAY || rc == VS_ERR_NONFINITE;
}

void warm_release(vs_warm_plan_t* p) {
  vs_plan_free(p->first);
  vs_plan_free(p->warm);
  cudaFree(p->x);
  cudaFree(p->y);
  delete p;
}

int warm_items(const vs_warm_plan_t* p, float* out, const float* init, const std::vector<int>& idx,
               std::vector<vs_batch_item>& items) {
  const size_t nn = (size_t)p->n * p->n;
  items.resize(idx.size());
  for (size_t j = 0; j < idx.size(); ++j) {
    const size_t o = (size_t)idx[j] * nn;
    items[j] = vs_batch_item{p->k, p->pd + o, p->pl + o, p->sk ? p->sk + o : nullptr, out + o,
                             init ? init + o : nullptr};
  }
  return VS_OK;
}

}  // namespace

extern "C" int vs_warm_plan_create(vs_kernel k, int count, const float* p_dyn, const float* p_leak0,
                                   const float* s_kappa, float* theta, float* theta1,
                                   float* theta_init, vs_model model,
                                   const vs_solve_params* params, vs_warm_plan* out,
                                   void* stream) {
  if (!out) return vs_set_error(VS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!k || !model || count < 1 || !p_dyn || !p_leak0 || !theta || !theta1 || !theta_init)
    return vs_set_error(VS_ERR_INVALID_ARG, "bad warm-plan arguments");
  const int n = k->n, R = model->R;
  if (R < 4 || n % R) return vs_set_error(VS_ERR_INVALID_ARG, "model resolution %d does not divide n %d", R, n);
  int rc = vs_validate_params(params);
  if (rc) return rc;
  vs_warm_plan_t* p = new vs_warm_plan_t();
  p->k = k;
  p->model = model;
  p->count = count;
  p->n = n;
  p->R = R;
  p->pd = p_dyn;
  p->pl = p_leak0;
  p->sk = s_kappa;
  p->theta = theta;
  p->theta1 = theta1;
  p->theta_init = theta_init;
  p->params = *params;
  rc = ensure_acts(model, std::min(count, 256));     // no allocation inside a run
  if (rc) {
    delete p;
    return rc;
  }
  cudaError_t e = cudaMalloc(&p->x, sizeof(float) * 3 * (size_t)R * R * count);
  if (e == cudaSuccess) e = cudaMalloc(&p->y, sizeof(float) * (size_t)R * R * count);
  if (e != cudaSuccess) {
    warm_release(p);
    return vs_set_error(e == cudaErrorMemoryAllocation ? VS_ERR_OOM : VS_ERR_CUDA,
                        "warm-plan buffers: %s", cudaGetErrorString(e));
  }
  std::vector<int> all(count);
  for (int i = 0; i < count; ++i) all[i] = i;
  std::vector<vs_batch_item> items;
  vs_solve_params one = *params;
  one.max_iter = 1;                                   // the first iterate only
  warm_items(p, theta1, nullptr, all, items);
  rc = vs_plan_create(items.data(), count, &one, &p->first, stream);
  if (rc == VS_OK) {
    warm_items(p, theta, theta_init, all, items);
    rc = vs_plan_create(items.data(), count, params, &p->warm, stream);
  }
  if (rc != VS_OK) {
    warm_release(p);
    return rc;
  }
  *out = p;
  return VS_OK;
}

extern "C" int vs_warm_plan_run(vs_warm_plan p, int stages, void* stream) {
  if (!p) return vs_set_error(VS_ERR_INVALID_ARG, "NULL warm plan");
  if (stages < 1 || stages > VS_WARM_ALL) return vs_set_error(VS_ERR_INVALID_ARG, "stages %d not in 1..7", stages);
  int rc = VS_OK;
  if (stages & VS_WARM_FIRST) rc = vs_plan_run(p->first, stream);
  if (rc == VS_OK && (stages & VS_WARM_PREDICT)) {
    rc = vs_warm_features(p->theta1, p->pl, p->sk, p->count, p->n, p->R, p->x, stream);
    if (rc == VS_OK) rc = vs_model_forward_tc(p->model, p->x, p->y, p->count, stream);
    if (rc == VS_OK)
      rc = vs_warm_apply(p->theta1, p->y, p->count, p->n, p->R, p->theta_init, stream);
  }
  if (rc == VS_OK && (stages & VS_WARM_SOLVE)) rc = vs_plan_run(p->warm, stream);
  return rc;
}

extern "C" int vs_warm_plan_launches(vs_warm_plan p) {
  if (!p) return 0;
  const int chunks = (p->count + 255) / 256;          // the network runs 256 maps at a time
  return vs_plan_launches(p->first) + 1 + 12 * chunks + 1 + vs_plan_launches(p->warm);
}

extern "C" int vs_warm_plan_info(vs_warm_plan p, vs_solve_info* info_host, int fallback,
                                 int* fell_back_host, void* stream) {
  if (!p || !info_host) return vs_set_error(VS_ERR_INVALID_ARG, "NULL warm plan or output");
  int rc = vs_plan_info(p->warm, info_host, stream);
  if (!per_map_status(rc)) return rc;                 // a launch-level error
  if (fell_back_host) memset(fell_back_host, 0, sizeof(int) * p->count);
  std::vector<int> bad;
  for (int i = 0; i < p->count; ++i)
    if (info_host[i].status != VS_OK) bad.push_back(i);
  if (!fallback || bad.empty()) return rc;
  // solve those maps again from theta_0 = 0
  std::vector<vs_batch_item> items;
  warm_items(p, p->theta, nullptr, bad, items);
  std::vector<vs_solve_info> redo(bad.size());
  int rc2 = vs_solve_batch(items.data(), (int)bad.size(), &p->params, redo.data(), stream);
  if (!per_map_status(rc2)) return rc2;
  int worst = VS_OK;
  for (size_t j = 0; j < bad.size(); ++j) {
    info_host[bad[j]] = redo[j];
    info_host[bad[j]].fell_back = 1;
    if (fell_back_host) fell_back_host[bad[j]] = 1;
  }
  for (int i = 0; i < p->count; ++i) worst = std::max(worst, info_host[i].status);
  return worst;
}

extern "C" void vs_warm_plan_free(vs_warm_plan p) {
  if (p) warm_release(p);
}
