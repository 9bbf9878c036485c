// One-shot closed form of the leakage/conductivity coupling (Sec. IV-C,
// Eqs. 21, 25 and 26), for a batch of maps of one kernel.
//
//   u = L_det * (P_dyn + P_leak0) + (P_leak0 - mu) . r,   theta = phi(u)
//   L_det = K~ / (1 - beta mu K~)                         (Eq. 21, alpha term dropped)
//   r     = beta L_det^2 * (P_dyn + P_leak0)              (Eq. 25 to first order, VS_CF_CONV)
//         = (beta L_det^2 * delta_centre) sum(P_dyn + P_leak0)   (Eq. 26 literally, VS_CF_IMPULSE)
// where * is the mirror-image convolution (diagonal in the DCT-II basis) and
// . the Hadamard product. One forward 2-D cosine transform and two inverse
// ones per map, in three launches over all maps:
//   rows : q = P_dyn + P_leak0, forward DCT along x, transposed store; per-task
//          partial sums of P_leak0 and q;
//   cols : forward DCT along y, both spectral multipliers, two inverse DCTs
//          along y;
//   rows : two inverse DCTs along x, Hadamard combination, phi;
// and a fourth, one thread per map, that writes the per-map outcome.
// Grids of 32^2 .. 256^2 take the cluster engine's closed-form instantiation
// instead (vs_cluster.cu): one thread-block cluster per map, the map and its
// spectra in shared memory, no spectral scratch in global memory.
#include <math.h>
#include <stdint.h>

#include <algorithm>
#include <mutex>

#include "vs_fft.cuh"
#include "vs_internal.cuh"
#include "vs_solve_common.cuh"

using namespace vsfft;

namespace {

constexpr int kCfThreads = 256;
constexpr int kCfRunaway = 1, kCfNonfinite = 2;

struct CfArgs {
  const float* p_dyn;    // [count][n][n]
  const float* p_leak0;
  const float* s;        // nullable
  float* theta;
  float* wa;             // [count][n][n] transposed spectral scratch (L_det part)
  float* wb;             // [count][n][n] (random part)
  double2* part;         // [count][tasks] (sum P_leak0, sum q) per row task
  int* flags;            // [count]
  vs_solve_info* info;   // [count]
  const float* Kt;       // [n][n]
  const float2* tw;      // 4n twiddles
  const int* dr;         // digit reversal
  float beta, alpha, kmax;
  int n, rb, tasks, count, mode;
};

__device__ __forceinline__ double2 block_sum2(double2 v, double2* red) {
  for (int o = 16; o > 0; o >>= 1) {
    v.x += __shfl_down_sync(0xffffffffu, v.x, o);
    v.y += __shfl_down_sync(0xffffffffu, v.y, o);
  }
  const int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double2 r = make_double2(0.0, 0.0);
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r.x += red[i].x, r.y += red[i].y;
  __syncthreads();
  return r;
}

__device__ __forceinline__ double map_mu(const CfArgs& a, int b, double* total) {
  double sl = 0.0, sq = 0.0;
  for (int i = 0; i < a.tasks; ++i) {
    const double2 v = a.part[(size_t)b * a.tasks + i];
    sl += v.x;
    sq += v.y;
  }
  if (total) *total = sq;
  return sl / ((double)a.n * a.n);
}

// Forward DCT along x of rows y0 .. y0 + rb - 1 held in buf (pairs of rows as
// float2, Makhoul order), stored transposed: W[k * n + y].
__device__ __forceinline__ void rows_forward_store(const CfArgs& a, float2* buf, float* W, int y0) {
  const int n = a.n, F = a.rb >> 1, NP = padded_len(n), half = n >> 1, lgF = __ffs(F) - 1;
  fft_forward(buf, n, F, NP, a.tw);
  for (int it = threadIdx.x; it < F * (half + 1); it += blockDim.x) {
    const int f = it & (F - 1), k = it >> lgF, nk = n - k;
    const float2 zk = buf[f * NP + pad(__ldg(&a.dr[k]))];
    const float2 znk = buf[f * NP + pad(__ldg(&a.dr[k == 0 ? 0 : nk]))];
    *reinterpret_cast<float2*>(W + (size_t)k * n + y0 + 2 * f) = dct_post(zk, znk, __ldg(&a.tw[k]));
    if (k != 0 && k != half)
      *reinterpret_cast<float2*>(W + (size_t)nk * n + y0 + 2 * f) = dct_post(znk, zk, __ldg(&a.tw[nk]));
  }
}

// Inverse DCT along x of rows y0 .. y0 + rb - 1 from the transposed spectra W
// into buf (natural Makhoul order afterwards).
__device__ __forceinline__ void rows_inverse_load(const CfArgs& a, float2* buf, const float* W, int y0) {
  const int n = a.n, F = a.rb >> 1, NP = padded_len(n), half = n >> 1, lgF = __ffs(F) - 1;
  for (int it = threadIdx.x; it < F * (half + 1); it += blockDim.x) {
    const int f = it & (F - 1), k = it >> lgF, nk = n - k;
    const float2 xk = *reinterpret_cast<const float2*>(W + (size_t)k * n + y0 + 2 * f);
    const float2 xnk = k ? *reinterpret_cast<const float2*>(W + (size_t)nk * n + y0 + 2 * f)
                         : make_float2(0.f, 0.f);
    buf[f * NP + pad(__ldg(&a.dr[k]))] = dct_pre(xk.x, xnk.x, xk.y, xnk.y, __ldg(&a.tw[k]));
    if (k != 0 && k != half)
      buf[f * NP + pad(__ldg(&a.dr[nk]))] = dct_pre(xnk.x, xk.x, xnk.y, xk.y, __ldg(&a.tw[nk]));
  }
  __syncthreads();
  fft_inverse(buf, n, F, NP, a.tw);
}

__global__ void __launch_bounds__(kCfThreads) k_cf_rows_fwd(CfArgs a) {
  extern __shared__ float2 sm[];
  __shared__ double2 red[kCfThreads / 32];
  const int b = blockIdx.x / a.tasks, chunk = blockIdx.x % a.tasks;
  const int n = a.n, F = a.rb >> 1, NP = padded_len(n), lgn = __ffs(n) - 1;
  const int y0 = chunk * a.rb;
  const size_t base = (size_t)b * n * n;
  double2 acc = make_double2(0.0, 0.0);
  for (int i = threadIdx.x; i < F * n; i += blockDim.x) {
    const int f = i >> lgn, x = i & (n - 1);
    const size_t i0 = base + (size_t)(y0 + 2 * f) * n + x, i1 = i0 + n;
    const float l0 = __ldg(&a.p_leak0[i0]), l1 = __ldg(&a.p_leak0[i1]);
    const float q0 = __ldg(&a.p_dyn[i0]) + l0, q1 = __ldg(&a.p_dyn[i1]) + l1;
    acc.x += (double)l0 + (double)l1;
    acc.y += (double)q0 + (double)q1;
    sm[f * NP + pad(makhoul_pos(x, n))] = make_float2(q0, q1);
  }
  const double2 tot = block_sum2(acc, red);
  if (threadIdx.x == 0) a.part[(size_t)b * a.tasks + chunk] = tot;
  __syncthreads();
  rows_forward_store(a, sm, a.wa + base, y0);
}

__global__ void __launch_bounds__(kCfThreads) k_cf_cols(CfArgs a) {
  extern __shared__ float2 sm[];
  const int b = blockIdx.x / a.tasks, chunk = blockIdx.x % a.tasks;
  const int n = a.n, F = a.rb >> 1, NP = padded_len(n), half = n >> 1;
  const int lgF = __ffs(F) - 1, lgn = __ffs(n) - 1;
  float2* sb = sm + F * NP;
  const int p0 = chunk * a.rb;
  const size_t base = (size_t)b * n * n;
  float* WA = a.wa + base;
  float* WB = a.wb + base;
  const float mu = (float)map_mu(a, b, nullptr);
  const float bm = a.beta * mu;
  if (chunk == 0 && threadIdx.x == 0 && (double)a.beta * mu * (double)a.kmax >= 0.999)
    atomicOr(&a.flags[b], kCfRunaway);
  for (int i = threadIdx.x; i < F * n; i += blockDim.x) {
    const int f = i >> lgn, j = i & (n - 1);
    sm[f * NP + pad(makhoul_pos(j, n))] =
        make_float2(WA[(size_t)(p0 + 2 * f) * n + j], WA[(size_t)(p0 + 2 * f + 1) * n + j]);
  }
  __syncthreads();
  fft_forward(sm, n, F, NP, a.tw);
  const float inv_n2 = 1.f / ((float)n * (float)n);
  const int c2 = n + 1;                   // 2c + 1 for the centre cell c = n / 2
  // 2-D DCT-II of a unit impulse at (c, c): cos(pi p (2c+1) / 2n) cos(pi k (2c+1) / 2n)
  auto dimp = [&](int p) { return cospif((float)((p * c2) % (4 * n)) / (float)(2 * n)); };
  // Per (k, n - k) pair a thread owns positions ia, ib of both buffers: the
  // L_det products go to sb, the random part replaces the spectrum in sm.
  for (int it = threadIdx.x; it < F * (half + 1); it += blockDim.x) {
    const int f = it & (F - 1), k = it >> lgF, nk = n - k;
    const int ia = f * NP + pad(__ldg(&a.dr[k]));
    const int ib = f * NP + pad(__ldg(&a.dr[k == 0 ? 0 : nk]));
    const float2 zk = sm[ia], znk = sm[ib];
    const float2 xk = dct_post(zk, znk, __ldg(&a.tw[k]));
    const float2 xnk = k ? dct_post(znk, zk, __ldg(&a.tw[nk])) : make_float2(0.f, 0.f);
    const int pa = p0 + 2 * f;            // x-frequencies of the two columns
    // multipliers of mode (x-frequency p, y-frequency kq) for spectrum value x
    auto mult = [&](int p, int kq, float x, float& va, float& vb) {
      const float K = __ldg(&a.Kt[(size_t)p * n + kq]);
      const float Ld = K / (1.f - bm * K);
      const float src = a.mode == VS_CF_IMPULSE ? dimp(p) * dimp(kq) : x;
      va = x * Ld * inv_n2;
      vb = src * a.beta * Ld * Ld * inv_n2;
    };
    float2 ak, bk, ank = make_float2(0.f, 0.f), bnk = make_float2(0.f, 0.f);
    mult(pa, k, xk.x, ak.x, bk.x);
    mult(pa + 1, k, xk.y, ak.y, bk.y);
    if (k != 0 && k != half) {
      mult(pa, nk, xnk.x, ank.x, bnk.x);
      mult(pa + 1, nk, xnk.y, ank.y, bnk.y);
    } else if (k == half) {
      ank = ak;
      bnk = bk;
    }
    sb[ia] = dct_pre(ak.x, ank.x, ak.y, ank.y, __ldg(&a.tw[k]));
    sm[ia] = dct_pre(bk.x, bnk.x, bk.y, bnk.y, __ldg(&a.tw[k]));
    if (k != 0 && k != half) {
      sb[ib] = dct_pre(ank.x, ak.x, ank.y, ak.y, __ldg(&a.tw[nk]));
      sm[ib] = dct_pre(bnk.x, bk.x, bnk.y, bk.y, __ldg(&a.tw[nk]));
    }
  }
  __syncthreads();
  fft_inverse(sb, n, F, NP, a.tw);
  fft_inverse(sm, n, F, NP, a.tw);
  for (int i = threadIdx.x; i < F * n; i += blockDim.x) {
    const int f = i >> lgn, j = i & (n - 1);
    const int pos = f * NP + pad(makhoul_pos(j, n));
    const float2 va = sb[pos], vb = sm[pos];
    WA[(size_t)(p0 + 2 * f) * n + j] = va.x;
    WA[(size_t)(p0 + 2 * f + 1) * n + j] = va.y;
    WB[(size_t)(p0 + 2 * f) * n + j] = vb.x;
    WB[(size_t)(p0 + 2 * f + 1) * n + j] = vb.y;
  }
}

__global__ void __launch_bounds__(kCfThreads) k_cf_rows_inv(CfArgs a) {
  extern __shared__ float2 sm[];
  __shared__ int red_flags;
  const int b = blockIdx.x / a.tasks, chunk = blockIdx.x % a.tasks;
  const int n = a.n, F = a.rb >> 1, NP = padded_len(n), lgn = __ffs(n) - 1;
  float2* sb = sm + F * NP;
  const int y0 = chunk * a.rb;
  const size_t base = (size_t)b * n * n;
  if (threadIdx.x == 0) red_flags = 0;
  rows_inverse_load(a, sm, a.wa + base, y0);
  rows_inverse_load(a, sb, a.wb + base, y0);
  double total = 0.0;
  const float mu = (float)map_mu(a, b, &total);
  const float scale = a.mode == VS_CF_IMPULSE ? (float)total : 1.f;
  int flags = 0;
  for (int i = threadIdx.x; i < F * n; i += blockDim.x) {
    const int f = i >> lgn, x = i & (n - 1);
    const int pos = f * NP + pad(makhoul_pos(x, n));
    const float2 ud = sm[pos], r = sb[pos];
#pragma unroll
    for (int h = 0; h < 2; ++h) {
      const size_t idx = base + (size_t)(y0 + 2 * f + h) * n + x;
      const float pv = __ldg(&a.p_leak0[idx]) - mu;
      const float u = fmaf(pv * scale, h ? r.y : r.x, h ? ud.y : ud.x);
      const float sk = a.s ? __ldg(&a.s[idx]) : 1.f;
      const float den = fmaf(-a.alpha * sk, u, 1.f);
      if (!(den > 0.05f)) flags |= kCfRunaway;
      const float th = sk * u / den;
      if (!isfinite(th)) flags |= kCfNonfinite;
      a.theta[idx] = th;
    }
  }
  if (flags) atomicOr(&red_flags, flags);
  __syncthreads();
  if (threadIdx.x == 0 && red_flags) atomicOr(&a.flags[b], red_flags);
}

__global__ void k_cf_info(CfArgs a) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= a.count) return;
  const int fl = a.flags[b];
  vs_solve_info inf;
  // a runaway map (beta mu max K >= 1, or 1 - alpha s u <= 0.05) is reported as
  // such even where its values also overflowed
  inf.status = (fl & kCfRunaway) ? VS_ERR_RUNAWAY : (fl & kCfNonfinite) ? VS_ERR_NONFINITE : VS_OK;
  inf.iterations = 0;
  inf.residual_K = 0.0;
  inf.mu_W = map_mu(a, b, nullptr);
  inf.fell_back = 0;
  a.info[b] = inf;
}

// Per-map descriptors of a contiguous batch for the cluster instantiation.
__global__ void k_cf_descs(vsk::MapDesc* maps, int* order, const float* p_dyn, const float* p_leak0,
                           const float* s, float* theta, const float* Kt, const float2* tw4n,
                           const int* digrev, float kmax, int n, int count) {
  const int b = blockIdx.x * blockDim.x + threadIdx.x;
  if (b >= count) return;
  const size_t off = (size_t)b * n * n;
  vsk::MapDesc m = {};
  m.p_dyn = p_dyn + off;
  m.p_leak0 = p_leak0 + off;
  m.s = s ? s + off : nullptr;
  m.theta = theta + off;
  m.Kt = Kt;
  m.tw4n = tw4n;
  m.digrev = digrev;
  m.kmax = kmax;
  m.n = n;
  maps[b] = m;
  order[b] = b;
}

size_t g_cf_smem_attr = 0;

}  // namespace

extern "C" int vs_solve_closed_form(vs_kernel k, int count, const float* p_dyn,
                                    const float* p_leak0, const float* s_kappa,
                                    const vs_solve_params* params, int mode, float* theta,
                                    vs_solve_info* info_host, void* stream) {
  if (!k) return vs_set_error(VS_ERR_INVALID_ARG, "NULL kernel");
  if (count < 1) return vs_set_error(VS_ERR_INVALID_ARG, "count %d < 1", count);
  if (!p_dyn || !p_leak0 || !theta) return vs_set_error(VS_ERR_INVALID_ARG, "NULL map");
  if (mode != VS_CF_CONV && mode != VS_CF_IMPULSE)
    return vs_set_error(VS_ERR_INVALID_ARG, "closed-form mode %d", mode);
  int rc = vs_validate_params(params);
  if (rc) return rc;
  if (vs_params_physics(params))
    return vs_set_error(VS_ERR_INVALID_ARG, "the closed form uses the linear models only");
  const uintptr_t al = (uintptr_t)p_dyn | (uintptr_t)p_leak0 | (uintptr_t)theta | (uintptr_t)s_kappa;
  if (al & 15u) return vs_set_error(VS_ERR_INVALID_ARG, "maps must be 16-byte aligned");
  const int n = k->n;
  cudaStream_t s = (cudaStream_t)stream;
  if (vsk::cluster_size_ok(n)) {
    // the cluster instantiation: descriptors, order and outcomes only
    void* scratch = nullptr;
    const size_t b_maps = sizeof(vsk::MapDesc) * (size_t)count;
    const size_t b_order = sizeof(int) * (size_t)count;
    const size_t b_info = sizeof(vs_solve_info) * (size_t)count;
    const size_t total = b_maps + b_order + b_info + 512;
    cudaError_t e = cudaMallocAsync(&scratch, total, s);
    if (e != cudaSuccess)
      return vs_set_error(e == cudaErrorMemoryAllocation ? VS_ERR_OOM : VS_ERR_CUDA,
                          "closed-form descriptors (%zu bytes): %s", total, cudaGetErrorString(e));
    char* p = (char*)scratch;
    vsk::MapDesc* maps = (vsk::MapDesc*)p;
    int* order = (int*)(p + ((b_maps + 255) & ~(size_t)255));
    vs_solve_info* info = (vs_solve_info*)((char*)order + ((b_order + 255) & ~(size_t)255) - 0);
    k_cf_descs<<<(count + 127) / 128, 128, 0, s>>>(maps, order, p_dyn, p_leak0, s_kappa, theta,
                                                   k->Kt32, k->fft->tw4n, k->fft->digrev, k->kmax,
                                                   n, count);
    e = cudaGetLastError();
    vsk::ClusterDev P = {};
    P.maps = maps;
    P.order = order;
    P.info = info;
    P.max_iter = 1;
    P.beta = (float)params->beta_per_K;
    P.alpha = (float)params->alpha_per_K;
    P.tol = (float)params->tol_K;
    P.cf_mode = mode;
    if (e == cudaSuccess) e = vsk::cluster_cf_launch(n, P, count, s);
    if (e == cudaSuccess && info_host)
      e = cudaMemcpyAsync(info_host, info, b_info, cudaMemcpyDeviceToHost, s);
    cudaError_t ef = cudaFreeAsync(scratch, s);
    if (e == cudaSuccess) e = ef;
    if (e != cudaSuccess) return vs_set_error(VS_ERR_CUDA, "closed form: %s", cudaGetErrorString(e));
    rc = VS_OK;
    if (info_host) {
      VS_CUDA_TRY(cudaStreamSynchronize(s));
      for (int i = 0; i < count; ++i) rc = std::max(rc, info_host[i].status);
    }
    return rc;
  }
  CfArgs a = {};
  a.p_dyn = p_dyn;
  a.p_leak0 = p_leak0;
  a.s = s_kappa;
  a.theta = theta;
  a.Kt = k->Kt32;
  a.tw = k->fft->tw4n;
  a.dr = k->fft->digrev;
  a.beta = (float)params->beta_per_K;
  a.alpha = (float)params->alpha_per_K;
  a.kmax = k->kmax;
  a.n = n;
  a.rb = std::max(2, std::min(n, std::min(64, 8192 / n)));
  a.tasks = n / a.rb;
  a.count = count;
  a.mode = mode;
  if ((size_t)count * a.tasks > 0x7fffffffu)
    return vs_set_error(VS_ERR_INVALID_ARG, "batch of %d maps is too large for one launch", count);
  const size_t nn = (size_t)n * n * count;
  const size_t smem = (size_t)2 * (a.rb / 2) * padded_len(n) * sizeof(float2);
  {
    static std::mutex mu;
    std::lock_guard<std::mutex> lk(mu);
    if (smem > g_cf_smem_attr) {
      VS_CUDA_TRY(cudaFuncSetAttribute(k_cf_rows_fwd, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      VS_CUDA_TRY(cudaFuncSetAttribute(k_cf_cols, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      VS_CUDA_TRY(cudaFuncSetAttribute(k_cf_rows_inv, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
      g_cf_smem_attr = smem;
    }
  }
  void* scratch = nullptr;
  const size_t bytes_w = nn * sizeof(float);
  const size_t bytes_part = sizeof(double2) * (size_t)count * a.tasks;
  const size_t bytes_total = 2 * bytes_w + bytes_part + sizeof(int) * count + sizeof(vs_solve_info) * count + 256;
  cudaError_t e = cudaMallocAsync(&scratch, bytes_total, s);
  if (e != cudaSuccess)
    return vs_set_error(e == cudaErrorMemoryAllocation ? VS_ERR_OOM : VS_ERR_CUDA,
                        "closed-form scratch (%zu bytes): %s", bytes_total, cudaGetErrorString(e));
  char* p = (char*)scratch;
  a.wa = (float*)p;
  a.wb = (float*)(p + bytes_w);
  a.part = (double2*)(p + 2 * bytes_w);
  a.info = (vs_solve_info*)(p + 2 * bytes_w + bytes_part);
  a.flags = (int*)((char*)a.info + sizeof(vs_solve_info) * count);
  rc = VS_OK;
  e = cudaMemsetAsync(a.flags, 0, sizeof(int) * count, s);
  const unsigned blocks = (unsigned)((size_t)count * a.tasks);
  if (e == cudaSuccess) {
    k_cf_rows_fwd<<<blocks, kCfThreads, smem, s>>>(a);
    k_cf_cols<<<blocks, kCfThreads, smem, s>>>(a);
    k_cf_rows_inv<<<blocks, kCfThreads, smem, s>>>(a);
    k_cf_info<<<(count + 127) / 128, 128, 0, s>>>(a);
    e = cudaGetLastError();
  }
  if (e == cudaSuccess && info_host)
    e = cudaMemcpyAsync(info_host, a.info, sizeof(vs_solve_info) * count, cudaMemcpyDeviceToHost, s);
  cudaError_t ef = cudaFreeAsync(scratch, s);
  if (e == cudaSuccess) e = ef;
  if (e != cudaSuccess) return vs_set_error(VS_ERR_CUDA, "closed form: %s", cudaGetErrorString(e));
  if (info_host) {
    VS_CUDA_TRY(cudaStreamSynchronize(s));
    for (int i = 0; i < count; ++i) rc = std::max(rc, info_host[i].status);
  }
  return rc;
}
