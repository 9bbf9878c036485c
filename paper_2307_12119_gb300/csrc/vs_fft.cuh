// Shared-memory FFT building blocks for the cosine-basis convolution.
//
// The mirror-image convolution of Sec. IV-F is diagonal in the DCT-II basis
// (the even extension of the map is what a DCT-II encodes). A length-n DCT-II
// of a real sequence is computed from a length-n complex FFT of the reordered
// sequence v[i] = x[2i], v[n-1-i] = x[2i+1] (Makhoul's reordering), two real
// sequences at a time packed as real and imaginary parts.
//
// The FFT is in place in shared memory: forward = decimation-in-frequency
// radix passes (natural order in, digit-reversed order out); inverse =
// the same passes undone in reverse order (digit-reversed in, natural out).
// Radix 16 passes first, then one radix-8/4/2 pass for the remaining factor.
// Complex index i of an FFT buffer is stored at i + (i >> 4) (one pad slot per
// 16) to spread the strided accesses of the late passes over banks, and
// consecutive FFTs of a buffer start an odd number of slots apart.
#pragma once

#include <cuda_runtime.h>

namespace vsfft {

__device__ __forceinline__ int pad(int i) { return i + (i >> 4); }
// Odd stride (in float2) between the FFTs of a buffer, so that the same
// element of consecutive FFTs falls in different banks.
__host__ __device__ inline int padded_len(int n) { return n + (n >> 4) + 1; }

__device__ __forceinline__ float2 cadd(float2 a, float2 b) { return make_float2(a.x + b.x, a.y + b.y); }
__device__ __forceinline__ float2 csub(float2 a, float2 b) { return make_float2(a.x - b.x, a.y - b.y); }
__device__ __forceinline__ float2 cmul(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, -a.y * b.y), fmaf(a.x, b.y, a.y * b.x));
}
// a * conj(b)
__device__ __forceinline__ float2 cmulc(float2 a, float2 b) {
  return make_float2(fmaf(a.x, b.x, a.y * b.y), fmaf(a.y, b.x, -a.x * b.y));
}
// multiply by -i (forward) or +i (inverse)
template <bool FWD>
__device__ __forceinline__ float2 rot90(float2 a) {
  return FWD ? make_float2(a.y, -a.x) : make_float2(-a.y, a.x);
}

template <bool FWD>
__device__ __forceinline__ void dft2(float2* v) {
  float2 a = v[0], b = v[1];
  v[0] = cadd(a, b);
  v[1] = csub(a, b);
}

template <bool FWD>
__device__ __forceinline__ void dft4(float2& x0, float2& x1, float2& x2, float2& x3) {
  float2 t0 = cadd(x0, x2), t1 = csub(x0, x2), t2 = cadd(x1, x3), t3 = rot90<FWD>(csub(x1, x3));
  x0 = cadd(t0, t2);
  x2 = csub(t0, t2);
  x1 = cadd(t1, t3);
  x3 = csub(t1, t3);
}

template <bool FWD>
__device__ __forceinline__ void dft4v(float2* v) { dft4<FWD>(v[0], v[1], v[2], v[3]); }

// W8^r = exp(-+2 pi i r / 8)
template <bool FWD>
__device__ __forceinline__ float2 w8(int r) {
  const float h = 0.70710678118654752440f;
  switch (r) {
    case 1: return FWD ? make_float2(h, -h) : make_float2(h, h);
    case 2: return FWD ? make_float2(0.f, -1.f) : make_float2(0.f, 1.f);
    case 3: return FWD ? make_float2(-h, -h) : make_float2(-h, h);
    default: return make_float2(1.f, 0.f);
  }
}

template <bool FWD>
__device__ __forceinline__ void dft8(float2* v) {
  // radix-2 split: a_r = x_r + x_{r+4}, b_r = (x_r - x_{r+4}) W8^r
  float2 a[4], b[4];
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    a[r] = cadd(v[r], v[r + 4]);
    b[r] = cmul(csub(v[r], v[r + 4]), w8<FWD>(r));
  }
  dft4v<FWD>(a);
  dft4v<FWD>(b);
#pragma unroll
  for (int k = 0; k < 4; ++k) {
    v[2 * k] = a[k];
    v[2 * k + 1] = b[k];
  }
}

// W16^j = exp(-+2 pi i j / 16), j in [0, 9]
template <bool FWD>
__device__ __forceinline__ float2 w16(int j) {
  const float c1 = 0.92387953251128675613f, s1 = 0.38268343236508977173f;
  const float h = 0.70710678118654752440f;
  float c, s;
  switch (j) {
    case 0: c = 1.f; s = 0.f; break;
    case 1: c = c1; s = s1; break;
    case 2: c = h; s = h; break;
    case 3: c = s1; s = c1; break;
    case 4: c = 0.f; s = 1.f; break;
    case 6: c = -h; s = h; break;
    case 9: c = -c1; s = -s1; break;
    default: c = 1.f; s = 0.f; break;
  }
  return FWD ? make_float2(c, -s) : make_float2(c, s);
}

template <bool FWD>
__device__ __forceinline__ void dft16(float2* v) {
  // n = n1 + 4 n2, k = 4 k1 + k2
#pragma unroll
  for (int n1 = 0; n1 < 4; ++n1) dft4<FWD>(v[n1], v[n1 + 4], v[n1 + 8], v[n1 + 12]);
  // now v[n1 + 4 k2] = inner DFT over n2; twiddle by W16^{n1 k2}
#pragma unroll
  for (int n1 = 1; n1 < 4; ++n1)
#pragma unroll
    for (int k2 = 1; k2 < 4; ++k2) v[n1 + 4 * k2] = cmul(v[n1 + 4 * k2], w16<FWD>(n1 * k2));
  float2 o[16];
#pragma unroll
  for (int k2 = 0; k2 < 4; ++k2) {
    float2 a0 = v[4 * k2], a1 = v[4 * k2 + 1], a2 = v[4 * k2 + 2], a3 = v[4 * k2 + 3];
    dft4<FWD>(a0, a1, a2, a3);
    o[k2] = a0;
    o[4 + k2] = a1;
    o[8 + k2] = a2;
    o[12 + k2] = a3;
  }
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = o[i];
}

template <int R, bool FWD>
__device__ __forceinline__ void dftR(float2* v) {
  if constexpr (R == 16) dft16<FWD>(v);
  else if constexpr (R == 8) dft8<FWD>(v);
  else if constexpr (R == 4) dft4v<FWD>(v);
  else dft2<FWD>(v);
}

// Twiddle load: through the read-only path from global memory, or a plain
// load when the table has been copied to shared memory (TW_SMEM).
template <bool TW_SMEM>
__device__ __forceinline__ float2 tw_load(const float2* __restrict__ p) {
  if constexpr (TW_SMEM) return *p;
  else return __ldg(p);
}

// One radix-R pass over `nfft` in-place FFTs of length n stored with padded
// stride `stride` in shared memory. Blocks of length L, sub-stride m = L/R.
// Forward (DIF): butterfly, then twiddle W_L^{j r}. Inverse: conjugate
// twiddle, then inverse butterfly (exact inverse of the forward pass, x R).
template <int R, bool FWD, bool TW_SMEM = false>
__device__ __forceinline__ void fft_pass(float2* buf, int n, int L, int nfft, int stride,
                                         const float2* __restrict__ tw4n, int tid, int nthr) {
  // all sizes are powers of two: index math by shifts and masks
  const int m = L / R;
  const int lg_m = __ffs(m) - 1;
  const int per_fft = n / R;
  const int lg_per = __ffs(per_fft) - 1;
  const int total = nfft * per_fft;
  const int tws = 4 * (n / L);
  for (int b = tid; b < total; b += nthr) {
    int f = b >> lg_per;
    int rem = b & (per_fft - 1);
    int blk = rem >> lg_m;
    int j = rem & (m - 1);
    float2* base = buf + f * stride;
    int i0 = blk * L + j;
    float2 v[R];
#pragma unroll
    for (int r = 0; r < R; ++r) v[r] = base[pad(i0 + r * m)];
    if (FWD) {
      dftR<R, true>(v);
      if (m > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmul(v[r], tw_load<TW_SMEM>(&tw4n[j * r * tws]));
      }
    } else {
      if (m > 1) {
#pragma unroll
        for (int r = 1; r < R; ++r) v[r] = cmulc(v[r], tw_load<TW_SMEM>(&tw4n[j * r * tws]));
      }
      dftR<R, false>(v);
    }
#pragma unroll
    for (int r = 0; r < R; ++r) base[pad(i0 + r * m)] = v[r];
  }
}

// Radix schedule: 16s first, then the remaining factor (8, 4 or 2).
__device__ __forceinline__ int n_passes(int n) {
  int p = 0;
  while (n >= 16) { n >>= 4; ++p; }
  return p + (n > 1 ? 1 : 0);
}
__device__ __forceinline__ int pass_radix(int n, int pass) {
  int rem = n;
  for (int i = 0; i < pass; ++i) rem /= (rem >= 16 ? 16 : rem);
  return rem >= 16 ? 16 : rem;
}

// Full forward FFT (natural -> digit-reversed), synchronising between passes.
template <bool TW_SMEM = false>
__device__ __forceinline__ void fft_forward(float2* buf, int n, int nfft, int stride,
                                            const float2* __restrict__ tw4n) {
  int L = n;
  const int np = n_passes(n);
  for (int p = 0; p < np; ++p) {
    int R = pass_radix(n, p);
    switch (R) {
      case 16: fft_pass<16, true, TW_SMEM>(buf, n, L, nfft, stride, tw4n, threadIdx.x, blockDim.x); break;
      case 8: fft_pass<8, true, TW_SMEM>(buf, n, L, nfft, stride, tw4n, threadIdx.x, blockDim.x); break;
      case 4: fft_pass<4, true, TW_SMEM>(buf, n, L, nfft, stride, tw4n, threadIdx.x, blockDim.x); break;
      default: fft_pass<2, true, TW_SMEM>(buf, n, L, nfft, stride, tw4n, threadIdx.x, blockDim.x); break;
    }
    L /= R;
    __syncthreads();
  }
}

// Full inverse FFT (digit-reversed -> natural, unnormalised), syncing.
template <bool TW_SMEM = false>
__device__ __forceinline__ void fft_inverse(float2* buf, int n, int nfft, int stride,
                                            const float2* __restrict__ tw4n) {
  const int np = n_passes(n);
  for (int p = np - 1; p >= 0; --p) {
    int R = pass_radix(n, p);
    int L = n;
    for (int i = 0; i < p; ++i) L /= pass_radix(n, i);
    switch (R) {
      case 16: fft_pass<16, false, TW_SMEM>(buf, n, L, nfft, stride, tw4n, threadIdx.x, blockDim.x); break;
      case 8: fft_pass<8, false, TW_SMEM>(buf, n, L, nfft, stride, tw4n, threadIdx.x, blockDim.x); break;
      case 4: fft_pass<4, false, TW_SMEM>(buf, n, L, nfft, stride, tw4n, threadIdx.x, blockDim.x); break;
      default: fft_pass<2, false, TW_SMEM>(buf, n, L, nfft, stride, tw4n, threadIdx.x, blockDim.x); break;
    }
    __syncthreads();
  }
}

// Position in the reordered sequence v of source sample j (Makhoul).
__device__ __forceinline__ int makhoul_pos(int j, int n) {
  return (j & 1) ? (n - 1 - (j >> 1)) : (j >> 1);
}

// Separation of two packed real sequences after the forward FFT, and the
// DCT-II post-twiddle: given Z[k], Z[n-k] (n-k taken mod n) returns
// (Xa[k], Xb[k]) with X[k] = Re(exp(-i pi k / 2n) V[k]).
__device__ __forceinline__ float2 dct_post(float2 zk, float2 znk, float2 w) {
  // w = exp(-i pi k / (2n)) = (c, -s)
  float c = w.x, s = -w.y;
  float ar = 0.5f * (zk.x + znk.x), ai = 0.5f * (zk.y - znk.y);
  float br = 0.5f * (zk.y + znk.y), bi = -0.5f * (zk.x - znk.x);
  return make_float2(fmaf(c, ar, s * ai), fmaf(c, br, s * bi));
}

// Inverse pre-twiddle: from real spectra pairs (Xa[k], Xa[n-k]) and
// (Xb[k], Xb[n-k]) (X[n] := 0) build Z[k] = Va[k] + i Vb[k] with
// V[k] = exp(i pi k / 2n) (X[k] - i X[n-k]).
__device__ __forceinline__ float2 dct_pre(float xak, float xank, float xbk, float xbnk, float2 w) {
  float c = w.x, s = -w.y;
  float var = fmaf(c, xak, s * xank), vai = fmaf(s, xak, -c * xank);
  float vbr = fmaf(c, xbk, s * xbnk), vbi = fmaf(s, xbk, -c * xbnk);
  return make_float2(var - vbi, vai + vbr);
}

}  // namespace vsfft
