// Green's-function build: stack spectrum, Hankel quadrature of the top-layer
// radial Green's function, fold of the image lattice, cosine transform and
// spectral sum of the spreader part (Sec. II-B Eq. 2, Sec. II-F Eq. 8,
// Appendix Theorem I, Sec. IV-F images).
//
// Split used (Sec. II-B decomposes the Green's function into a part that decays
// fast with r and a part carried by the heat spreader):
//   g(k)  = g1(k) + R(k),  g1(k) = tanh(k t0) / (kappa0 k)
// g1 is the source layer on an isothermal base; its radial function G1(r)
// decays like K0(pi r / 2 t0) and is summed over the image lattice in real
// space. R(k) = Z1 sech^2(k t0) / (1 + kappa0 k tanh(k t0) Z1) decays like
// exp(-2 k t0) and its lattice is summed in the spectral domain.
//
// Every cell is a uniform disc source of the cell's area, radius
// a = cell / sqrt(pi), with spectrum D(ka) = 2 J1(ka)/(ka). With the 2-D
// Fourier transform equal to 2 pi times the Hankel transform (Theorem I):
//   G1(r) = (1/2pi) int_0^inf g1(k) D(ka) J0(kr) k dk
//         = Ghs(r) - (1/(2 pi kappa0)) int_0^inf (1 - tanh(k t0)) D(ka) J0(kr) dk
// where Ghs is the disc on a half-space (closed form below). The remaining
// integrand decays like exp(-2 k t0), so a single Gauss-Legendre rule on
// [0, Kmax] with FP64 weights resolves it at every lattice radius.
#include <math.h>
#include <stdio.h>
#include <stdlib.h>

#include <algorithm>
#include <vector>

#include "vs_internal.cuh"

namespace {

constexpr double kPi = 3.141592653589793238462643383279502884;

// ------------------------------------------------------------ device physics

__device__ double tanhc_d(double x) {
  double ax = fabs(x);
  if (ax < 1e-6) return 1.0 - x * x / 3.0;
  return tanh(x) / x;
}

// Impedance looking down from the top of layer `first` (Eq. 1 per wavenumber).
__device__ double impedance_d(double k, const vs_stack_dev& st, int first) {
  double Z = 1.0 / st.h;
  for (int i = st.n_layers - 1; i >= first; --i) {
    double kt = k * st.t[i];
    double tau = tanh(kt);
    double series = st.t[i] / st.kappa[i] * tanhc_d(kt);
    Z = (Z + series) / (1.0 + st.kappa[i] * k * tau * Z);
  }
  return Z;
}

__device__ double ghat_d(double k, const vs_stack_dev& st) { return impedance_d(k, st, 0); }

// R(k) = g(k) - g1(k) without cancellation.
__device__ double grest_d(double k, const vs_stack_dev& st) {
  double x = k * st.t[0];
  if (x > 40.0) return 0.0;
  double Z1 = st.n_layers > 1 ? impedance_d(k, st, 1) : 1.0 / st.h;
  double c = cosh(x);
  return Z1 / (c * c) / (1.0 + st.kappa[0] * k * tanh(x) * Z1);
}

__device__ double disc_d(double x) {
  if (x < 1e-4) return 1.0 - x * x / 8.0;
  return 2.0 * j1(x) / x;
}

// Complete elliptic integrals K(m), E(m) (parameter m = modulus^2) by the
// arithmetic-geometric mean (Gauss).
__device__ void ellip_ke(double m, double* K, double* E) {
  double a = 1.0, b = sqrt(1.0 - m), c = sqrt(m);
  double sum = 0.5 * c * c, pw = 0.5;
  for (int it = 0; it < 40 && fabs(c) > 1e-17; ++it) {
    double an = 0.5 * (a + b);
    double bn = sqrt(a * b);
    c = 0.5 * (a - b);
    a = an;
    b = bn;
    pw *= 2.0;
    sum += pw * c * c;
  }
  *K = kPi / (2.0 * a);
  *E = *K * (1.0 - sum);
}

// Unit-power uniform disc (radius a) on a half-space of conductivity kappa:
// source-plane temperature at distance r.
//   r = 0      : 1/(pi kappa a)
//   0 < r <= a : (2/(pi^2 kappa a)) E((r/a)^2)
//   r > a      : F(1/2,1/2;2;(a/r)^2) / (2 pi kappa r)   (Weber-Schafheitlin)
// The hypergeometric series is used for (a/r)^2 <= 1/2, the elliptic form
// 2r/(pi^2 kappa a^2) [E(m) - (1-m) K(m)], m = (a/r)^2, above.
__device__ double halfspace_disc_d(double r, double kappa, double a) {
  if (r == 0.0) return 1.0 / (kPi * kappa * a);
  if (r <= a) {
    double K, E;
    ellip_ke((r / a) * (r / a), &K, &E);
    return 2.0 / (kPi * kPi * kappa * a) * E;
  }
  double m = (a / r) * (a / r);
  if (m <= 0.5) {
    double term = 1.0, sum = 1.0;
    for (int n = 0; n < 200; ++n) {
      double hn = 0.5 + n;
      term *= hn * hn / ((2.0 + n) * (1.0 + n)) * m;
      sum += term;
      if (term < 1e-18 * sum) break;
    }
    return sum / (2.0 * kPi * kappa * r);
  }
  double K, E;
  ellip_ke(m, &K, &E);
  return 2.0 * r / (kPi * kPi * kappa * a * a) * (E - (1.0 - m) * K);
}

// ------------------------------------------------------------ kernels

// w'_i = w_i * (1 - tanh(k_i t0)) * D(k_i a) / (2 pi kappa0), FP64.
__global__ void k_quad_weights(const double* __restrict__ x, const double* __restrict__ w,
                               int nq, double kmax, vs_stack_dev st, double a,
                               double* __restrict__ kq, double* __restrict__ wq) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= nq) return;
  double k = 0.5 * kmax * (x[i] + 1.0);
  double kt = k * st.t[0];
  double one_m_tanh = 2.0 * exp(-2.0 * kt) / (1.0 + exp(-2.0 * kt));
  kq[i] = k;
  wq[i] = 0.5 * kmax * w[i] * one_m_tanh * disc_d(k * a) / (2.0 * kPi * st.kappa[0]);
}

// One warp per radius: G1(r) = Ghs(r) - sum_i wq_i J0(kq_i r). FP64.
__global__ void k_hankel_radial(const double* __restrict__ r, int count,
                                const double* __restrict__ kq, const double* __restrict__ wq,
                                int nq, double kappa0, double a, double* __restrict__ out) {
  int warp = (blockIdx.x * blockDim.x + threadIdx.x) >> 5;
  int lane = threadIdx.x & 31;
  if (warp >= count) return;
  double rr = r[warp];
  double acc = 0.0;
  for (int i = lane; i < nq; i += 32) acc += wq[i] * j0(kq[i] * rr);
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if (lane == 0) out[warp] = halfspace_disc_d(rr, kappa0, a) - acc;
}

__global__ void k_scatter_radial(const int* __restrict__ mlist, const double* __restrict__ g,
                                 int count, double* __restrict__ table) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) table[mlist[i]] = g[i];
}

__global__ void k_radii(const int* __restrict__ mlist, int count, double cell,
                        double* __restrict__ r) {
  int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < count) r[i] = cell * sqrt((double)mlist[i]);
}

// Fold of the image lattice onto the 2n-periodic grid, quarter by symmetry:
// kper[dy][dx] = sum over lattice points (dx + 2n i, dy + 2n j) within the
// cutoff of G1, for dx, dy in [0, n].
__global__ void k_fold(const double* __restrict__ table, int m_max, int R, int n,
                       double* __restrict__ kper) {
  int dx = blockIdx.x * blockDim.x + threadIdx.x;
  int dy = blockIdx.y;
  if (dx > n || dy > n) return;
  int n2 = 2 * n;
  double acc = 0.0;
  int i0 = -((R + dx) / n2), i1 = (R - dx) / n2;
  int j0_ = -((R + dy) / n2), j1_ = (R - dy) / n2;
  for (int j = j0_; j <= j1_; ++j) {
    long long y = dy + (long long)n2 * j;
    for (int i = i0; i <= i1; ++i) {
      long long x = dx + (long long)n2 * i;
      long long m = x * x + y * y;
      if (m <= m_max) acc += table[m];
    }
  }
  kper[(size_t)dy * (n + 1) + dx] = acc;
}

// Cosine transform of an even 2n-periodic sequence known on [0, n]:
// sum_{d=0}^{2n-1} f(d) cos(pi q d / n) = f(0) + (-1)^q f(n) + 2 sum_{d=1}^{n-1} f(d) cos(..)
// Only d <= dmax can be non-zero. Pass over the last index:
//   out[row][q] = sum_d c_d in[row][d] cos(pi q d / n),  in row stride n+1.
__global__ void k_cos_rows(const double* __restrict__ in, int rows, int n, int dmax,
                           const double* __restrict__ cos2n, double* __restrict__ out) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  int row = blockIdx.y;
  if (q >= n || row >= rows) return;
  const double* f = in + (size_t)row * (n + 1);
  int n2 = 2 * n;
  double acc = f[0];
  int dlim = min(dmax, n - 1);
  for (int d = 1; d <= dlim; ++d) acc += 2.0 * f[d] * cos2n[(q * d) % n2];
  if (dmax >= n) acc += ((q & 1) ? -1.0 : 1.0) * f[n];
  out[(size_t)row * n + q] = acc;
}

// Second pass over the first index (rows of T are d, columns q):
//   K1[p][q] = sum_d c_d T[d][q] cos(pi p d / n)
__global__ void k_cos_cols(const double* __restrict__ T, int n, int dmax,
                           const double* __restrict__ cos2n, double* __restrict__ K1) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  int p = blockIdx.y;
  if (q >= n || p >= n) return;
  int n2 = 2 * n;
  double acc = T[q];
  int dlim = min(dmax, n - 1);
  for (int d = 1; d <= dlim; ++d) acc += 2.0 * T[(size_t)d * n + q] * cos2n[(p * d) % n2];
  if (dmax >= n) acc += ((p & 1) ? -1.0 : 1.0) * T[(size_t)n * n + q];
  K1[(size_t)p * n + q] = acc;
}

__global__ void k_cos_table(int n, double* __restrict__ c) {
  int j = blockIdx.x * blockDim.x + threadIdx.x;
  if (j < 2 * n) c[j] = cospi((double)j / (double)n);
}

// ------------------------------------------------------------ wider spreader
// Footprint-mean impedance of the spreader layers (first .. M-1) when they are
// a square of side Ls centred under the die of side L (Sec. II-B: the spreader
// carries a constant part of the Green's function). Cosine series of the wide
// layers: with d_m = (1/L) int_a^{a+L} cos(m pi x / Ls) dx (a = (Ls - L)/2,
// d_0 = 1) and w_m = eps_m (L / Ls) d_m^2 (eps_0 = 1, else 2), the mean rise
// over the footprint per unit flux is sum_{m,n} w_m w_n Z(pi sqrt(m^2+n^2)/Ls).
// Partial sums over m, n < M and m, n < M/2 per block, in a fixed order.
constexpr int kSprTerms = 2048;   // modes per axis (even)
constexpr int kSprBlocks = 128;
constexpr int kSprThreads = 256;

__device__ double spr_w(int m, double L, double Ls) {
  if (m == 0) return L / Ls;
  const double a = 0.5 * (Ls - L);
  const double d = Ls / ((double)m * kPi * L) *
                   (sin((double)m * kPi * (a + L) / Ls) - sin((double)m * kPi * a / Ls));
  return 2.0 * (L / Ls) * d * d;
}

__global__ void __launch_bounds__(kSprThreads) k_spreader_partial(vs_stack_dev st, double L,
                                                                  double* __restrict__ part) {
  __shared__ double red[2][kSprThreads];
  __shared__ double w[kSprTerms];
  const double Ls = st.spreader_side;
  for (int m = threadIdx.x; m < kSprTerms; m += kSprThreads) w[m] = spr_w(m, L, Ls);
  __syncthreads();
  double full = 0.0, half = 0.0;
  const long long total = (long long)kSprTerms * kSprTerms;
  for (long long i = (long long)blockIdx.x * kSprThreads + threadIdx.x; i < total;
       i += (long long)kSprBlocks * kSprThreads) {
    const int m = (int)(i / kSprTerms), n = (int)(i % kSprTerms);
    const double wm = w[m], wn = w[n];
    if (wm == 0.0 || wn == 0.0) continue;
    const double k = kPi * sqrt((double)m * m + (double)n * n) / Ls;
    const double v = wm * wn * impedance_d(k, st, st.spreader_layer);
    full += v;
    if (m < kSprTerms / 2 && n < kSprTerms / 2) half += v;
  }
  red[0][threadIdx.x] = full;
  red[1][threadIdx.x] = half;
  __syncthreads();
  for (int s = kSprThreads / 2; s > 0; s >>= 1) {
    if (threadIdx.x < s) {
      red[0][threadIdx.x] += red[0][threadIdx.x + s];
      red[1][threadIdx.x] += red[1][threadIdx.x + s];
    }
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    part[2 * blockIdx.x] = red[0][0];
    part[2 * blockIdx.x + 1] = red[1][0];
  }
}

// g^ of the uniform mode with the wide spreader: the die layers in series over
// the footprint-mean impedance, its 1/M^2 series tail removed by one
// Richardson step (4 S_M - S_{M/2}) / 3. Single thread, fixed order.
__global__ void k_spreader_g0(vs_stack_dev st, const double* __restrict__ part,
                              double* __restrict__ g0w) {
  if (blockIdx.x != 0 || threadIdx.x != 0) return;
  double full = 0.0, half = 0.0;
  for (int b = 0; b < kSprBlocks; ++b) {
    full += part[2 * b];
    half += part[2 * b + 1];
  }
  double top = 0.0;
  for (int i = 0; i < st.spreader_layer; ++i) top += st.t[i] / st.kappa[i];
  *g0w = top + (4.0 * full - half) / 3.0;
}

// Spectral part: cell^-2 sum_{s,t in [-S,S]} R(|k|) D(|k| a),
// k = pi (p + 2 n s, q + 2 n t) / L; added to K1 and converted to FP32.
// Also the transient tables for the primary mode when dt > 0. With a wider
// spreader (g0w != NULL) the uniform mode's primary term g^(0) / cell^2 takes
// g0w instead, in K and in the transient tables.
__global__ void k_spectral(const double* __restrict__ K1, int n, double L, int S,
                           vs_stack_dev st, double a, double dt,
                           double* __restrict__ K64, float* __restrict__ K32,
                           float* __restrict__ trA, float* __restrict__ trRho,
                           const double* __restrict__ g0w) {
  int q = blockIdx.x * blockDim.x + threadIdx.x;
  int p = blockIdx.y;
  if (q >= n || p >= n) return;
  double cell = L / n;
  double acc = 0.0;
  double kcut = 40.0 / st.t[0];
  for (int s = -S; s <= S; ++s) {
    double ky = kPi * (double)(p + 2 * n * s) / L;
    if (fabs(ky) > kcut) continue;
    for (int t = -S; t <= S; ++t) {
      double kx = kPi * (double)(q + 2 * n * t) / L;
      double kk = sqrt(ky * ky + kx * kx);
      if (kk > kcut) continue;
      acc += grest_d(kk, st) * disc_d(kk * a);
    }
  }
  size_t idx = (size_t)p * n + q;
  double v = K1[idx] + acc / (cell * cell);
  const bool wide = g0w != nullptr && idx == 0;
  if (wide) v += (*g0w - ghat_d(0.0, st)) / (cell * cell);
  K64[idx] = v;
  K32[idx] = (float)v;
  if (trA != nullptr) {
    double k0 = kPi * sqrt((double)p * p + (double)q * q) / L;
    double g = wide ? *g0w : ghat_d(k0, st);
    trA[idx] = (float)(g * disc_d(k0 * a) / (cell * cell));
    trRho[idx] = (float)exp(-dt / (st.heat_cap * g));
  }
}

// ------------------------------------------------------------ host helpers

// Gauss-Legendre nodes/weights on [-1, 1] by Newton iteration on the
// three-term recurrence of the Legendre polynomials.
void gauss_legendre(int n, std::vector<double>& x, std::vector<double>& w) {
  x.assign(n, 0.0);
  w.assign(n, 0.0);
  for (int i = 0; i < (n + 1) / 2; ++i) {
    double z = cos(kPi * (i + 0.75) / (n + 0.5));
    double dp = 1.0;
    for (int it = 0; it < 100; ++it) {
      double p0 = 1.0, p1 = z;
      for (int j = 2; j <= n; ++j) {
        double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
        p0 = p1;
        p1 = p2;
      }
      dp = n * (z * p1 - p0) / (z * z - 1.0);
      double dz = p1 / dp;
      z -= dz;
      if (fabs(dz) < 1e-16) {
        // one more evaluation at the converged point for the weight
        p0 = 1.0;
        p1 = z;
        for (int j = 2; j <= n; ++j) {
          double p2 = ((2.0 * j - 1.0) * z * p1 - (j - 1.0) * p0) / j;
          p0 = p1;
          p1 = p2;
        }
        dp = n * (z * p1 - p0) / (z * z - 1.0);
        break;
      }
    }
    x[i] = -z;
    x[n - 1 - i] = z;
    w[i] = w[n - 1 - i] = 2.0 / ((1.0 - z * z) * dp * dp);
  }
}

// Quadrature rule (device) for the remainder integral of G1.
struct QuadRule {
  double* kq = nullptr;
  double* wq = nullptr;
  int nq = 0;
};

int make_quad_rule(const vs_stack_dev& st, double a, int nq, cudaStream_t s, QuadRule* q) {
  std::vector<double> x, w;
  gauss_legendre(nq, x, w);
  // (1 - tanh(k t0)) < 1e-17 beyond k t0 = 20
  double kmax = 20.0 / st.t[0];
  double *dx = nullptr, *dw = nullptr;
  VS_CUDA_TRY(cudaMallocAsync(&dx, sizeof(double) * nq, s));
  VS_CUDA_TRY(cudaMallocAsync(&dw, sizeof(double) * nq, s));
  VS_CUDA_TRY(cudaMallocAsync(&q->kq, sizeof(double) * nq, s));
  VS_CUDA_TRY(cudaMallocAsync(&q->wq, sizeof(double) * nq, s));
  VS_CUDA_TRY(cudaMemcpyAsync(dx, x.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, s));
  VS_CUDA_TRY(cudaMemcpyAsync(dw, w.data(), sizeof(double) * nq, cudaMemcpyHostToDevice, s));
  k_quad_weights<<<(nq + 127) / 128, 128, 0, s>>>(dx, dw, nq, kmax, st, a, q->kq, q->wq);
  VS_CUDA_TRY(cudaGetLastError());
  // the host vectors must stay alive until the copies are done
  VS_CUDA_TRY(cudaStreamSynchronize(s));
  VS_CUDA_TRY(cudaFreeAsync(dx, s));
  VS_CUDA_TRY(cudaFreeAsync(dw, s));
  q->nq = nq;
  return VS_OK;
}

void free_quad_rule(QuadRule* q, cudaStream_t s) {
  if (q->kq) cudaFreeAsync(q->kq, s);
  if (q->wq) cudaFreeAsync(q->wq, s);
  q->kq = q->wq = nullptr;
}

}  // namespace

// ------------------------------------------------------------------ API glue

int vs_hankel_eval(const vs_stack_dev& st, double cell_m, int quad_nodes,
                   const double* r_dev, double* out_dev, int count, cudaStream_t s) {
  if (count <= 0) return VS_OK;
  double a = cell_m / sqrt(kPi);
  QuadRule q;
  int rc = make_quad_rule(st, a, quad_nodes, s, &q);
  if (rc != VS_OK) {
    free_quad_rule(&q, s);
    return rc;
  }
  int threads = 256;
  long long blocks = ((long long)count * 32 + threads - 1) / threads;
  k_hankel_radial<<<(unsigned)blocks, threads, 0, s>>>(r_dev, count, q.kq, q.wq, q.nq,
                                                      st.kappa[0], a, out_dev);
  cudaError_t e = cudaGetLastError();
  free_quad_rule(&q, s);
  if (e != cudaSuccess) return vs_set_error(VS_ERR_CUDA, "hankel launch: %s", cudaGetErrorString(e));
  return VS_OK;
}

extern "C" int vs_hankel_radial(const vs_stack* stack, const vs_grid* grid, int quad_nodes,
                                const double* r_dev, double* out_dev, int count, void* stream) {
  int rc = vs_validate_stack(stack);
  if (rc) return rc;
  if ((rc = vs_validate_grid(grid))) return rc;
  if (quad_nodes == 0) quad_nodes = 256;
  if (quad_nodes < 64 || quad_nodes > 1024)
    return vs_set_error(VS_ERR_INVALID_ARG, "quad_nodes %d outside [64, 1024]", quad_nodes);
  if (count < 0 || (count > 0 && (!r_dev || !out_dev)))
    return vs_set_error(VS_ERR_INVALID_ARG, "bad radius/output arrays");
  vs_stack_dev st;
  vs_stack_to_dev(stack, &st);
  return vs_hankel_eval(st, grid->die_m / grid->n, quad_nodes, r_dev, out_dev, count,
                        (cudaStream_t)stream);
}

static void free_kernel_arrays(vs_kernel_t* k) {
  if (!k) return;
  cudaFree(k->Kt64);
  cudaFree(k->Kt32);
  cudaFree(k->radial);
  cudaFree(k->trA);
  cudaFree(k->trRho);
}

extern "C" void vs_free_kernel(vs_kernel k) {
  if (!k) return;
  free_kernel_arrays(k);
  delete k;
}

extern "C" int vs_kernel_n(vs_kernel k) { return k ? k->n : -1; }

extern "C" int vs_make_kernel(const vs_stack* stack, const vs_grid* grid,
                              const vs_kernel_opts* opts, vs_kernel* out, void* stream) {
  if (!out) return vs_set_error(VS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  int rc = vs_validate_stack(stack);
  if (rc) return rc;
  if ((rc = vs_validate_grid(grid))) return rc;
  int nq = (opts && opts->quad_nodes) ? opts->quad_nodes : 256;
  double rel = (opts && opts->rel_tol > 0) ? opts->rel_tol : 1e-13;
  double dt = opts ? opts->dt_s : 0.0;
  if (nq < 64 || nq > 1024) return vs_set_error(VS_ERR_INVALID_ARG, "quad_nodes %d outside [64, 1024]", nq);
  if (rel < 1e-16 || rel > 1e-6) return vs_set_error(VS_ERR_INVALID_ARG, "rel_tol %g outside [1e-16, 1e-6]", rel);
  if (!(dt >= 0.0) || !isfinite(dt)) return vs_set_error(VS_ERR_INVALID_ARG, "dt_s must be >= 0");
  if (dt > 0.0 && !(stack->heat_cap_J_m2K > 0.0))
    return vs_set_error(VS_ERR_INVALID_ARG, "heat_cap_J_m2K must be > 0 for a transient kernel");
  const bool wide = stack->spreader_layer > 0 && stack->spreader_side_m != grid->die_m;
  if (stack->spreader_layer > 0 && !(stack->spreader_side_m >= grid->die_m))
    return vs_set_error(VS_ERR_INVALID_ARG, "spreader_side_m %g is smaller than the die (%g)",
                        stack->spreader_side_m, grid->die_m);

  cudaStream_t s = (cudaStream_t)stream;
  int n = grid->n;
  double L = grid->die_m;
  double cell = L / n;
  double a = cell / sqrt(kPi);

  vs_kernel_t* k = new vs_kernel_t();
  k->n = n;
  k->die_m = L;
  vs_stack_to_dev(stack, &k->st);
  k->quad_nodes = nq;
  k->rel_tol = rel;
  k->dt = dt;
  int fst = VS_OK;
  k->fft = vs_get_fft_tables(n, &fst);
  if (!k->fft) {
    delete k;
    return fst;
  }

  // real-space cutoff: G1 ~ K0(pi r / 2 t0) below rel beyond rc
  double t0 = k->st.t[0];
  double rcut = 2.0 * t0 / kPi * log(1.0 / rel) + 2.0 * t0;
  int R = (int)ceil(rcut / cell);
  long long mmax_ll = (long long)R * R;
  if (mmax_ll > 200000000LL) {
    delete k;
    return vs_set_error(VS_ERR_INVALID_ARG, "real-space cutoff too large (%d cells)", R);
  }
  int m_max = (int)mmax_ll;
  k->m_max = m_max;

  // unique squared radii i^2 + j^2 <= m_max (0 <= j <= i)
  std::vector<char> mark((size_t)m_max + 1, 0);
  for (long long i = 0; i <= R; ++i)
    for (long long j = 0; j <= i && i * i + j * j <= m_max; ++j) mark[i * i + j * j] = 1;
  std::vector<int> mlist;
  for (int m = 0; m <= m_max; ++m)
    if (mark[m]) mlist.push_back(m);
  int nu = (int)mlist.size();

  // alias rings of the spectral part: exp(-2 k t0) below rel
  int S = (int)ceil((cell * log(1.0 / rel) / (2.0 * kPi * t0) + 1.0) / 2.0) + 1;

  int* d_mlist = nullptr;
  double *d_r = nullptr, *d_g = nullptr, *d_kper = nullptr, *d_T = nullptr, *d_K1 = nullptr,
         *d_cos = nullptr, *d_spr = nullptr;
  QuadRule q;
  auto fail = [&](int code) {
    cudaStreamSynchronize(s);
    cudaFree(d_mlist);
    cudaFree(d_r);
    cudaFree(d_g);
    cudaFree(d_kper);
    cudaFree(d_T);
    cudaFree(d_K1);
    cudaFree(d_cos);
    cudaFree(d_spr);
    free_quad_rule(&q, s);
    free_kernel_arrays(k);
    delete k;
    return code;
  };
#define VS_BUILD_TRY(call)                                                              \
  do {                                                                                   \
    cudaError_t e_ = (call);                                                             \
    if (e_ != cudaSuccess)                                                               \
      return fail(vs_set_error(e_ == cudaErrorMemoryAllocation ? VS_ERR_OOM : VS_ERR_CUDA, \
                               "%s: %s", #call, cudaGetErrorString(e_)));               \
  } while (0)

  size_t nn = (size_t)n * n;
  VS_BUILD_TRY(cudaMalloc(&k->Kt64, nn * sizeof(double)));
  VS_BUILD_TRY(cudaMalloc(&k->Kt32, nn * sizeof(float)));
  VS_BUILD_TRY(cudaMalloc(&k->radial, ((size_t)m_max + 1) * sizeof(double)));
  if (dt > 0) {
    VS_BUILD_TRY(cudaMalloc(&k->trA, nn * sizeof(float)));
    VS_BUILD_TRY(cudaMalloc(&k->trRho, nn * sizeof(float)));
  }
  VS_BUILD_TRY(cudaMalloc(&d_mlist, sizeof(int) * nu));
  VS_BUILD_TRY(cudaMalloc(&d_r, sizeof(double) * nu));
  VS_BUILD_TRY(cudaMalloc(&d_g, sizeof(double) * nu));
  VS_BUILD_TRY(cudaMalloc(&d_kper, sizeof(double) * (n + 1) * (n + 1)));
  VS_BUILD_TRY(cudaMalloc(&d_T, sizeof(double) * (n + 1) * n));
  VS_BUILD_TRY(cudaMalloc(&d_K1, sizeof(double) * nn));
  VS_BUILD_TRY(cudaMalloc(&d_cos, sizeof(double) * 2 * n));
  if (wide) VS_BUILD_TRY(cudaMalloc(&d_spr, sizeof(double) * (2 * kSprBlocks + 1)));
  VS_BUILD_TRY(cudaMemsetAsync(k->radial, 0, ((size_t)m_max + 1) * sizeof(double), s));
  VS_BUILD_TRY(cudaMemcpyAsync(d_mlist, mlist.data(), sizeof(int) * nu, cudaMemcpyHostToDevice, s));

  // 1-2: quadrature rule and radial table
  int qrc = make_quad_rule(k->st, a, nq, s, &q);
  if (qrc != VS_OK) return fail(qrc);
  k_radii<<<(nu + 255) / 256, 256, 0, s>>>(d_mlist, nu, cell, d_r);
  {
    long long blocks = ((long long)nu * 32 + 255) / 256;
    k_hankel_radial<<<(unsigned)blocks, 256, 0, s>>>(d_r, nu, q.kq, q.wq, q.nq, k->st.kappa[0], a, d_g);
  }
  k_scatter_radial<<<(nu + 255) / 256, 256, 0, s>>>(d_mlist, d_g, nu, k->radial);
  VS_BUILD_TRY(cudaGetLastError());

  // 3: fold + cosine transform
  dim3 gf((n + 1 + 127) / 128, n + 1);
  k_fold<<<gf, 128, 0, s>>>(k->radial, m_max, R, n, d_kper);
  k_cos_table<<<(2 * n + 255) / 256, 256, 0, s>>>(n, d_cos);
  int dmax = std::min(n, R);
  dim3 gr((n + 127) / 128, n + 1);
  k_cos_rows<<<gr, 128, 0, s>>>(d_kper, n + 1, n, dmax, d_cos, d_T);
  dim3 gc((n + 127) / 128, n);
  k_cos_cols<<<gc, 128, 0, s>>>(d_T, n, dmax, d_cos, d_K1);
  // 4: the wider spreader's uniform mode, spectral part, FP32 copy, transient tables
  const double* g0w = nullptr;
  if (wide) {
    k_spreader_partial<<<kSprBlocks, kSprThreads, 0, s>>>(k->st, L, d_spr + 1);
    k_spreader_g0<<<1, 1, 0, s>>>(k->st, d_spr + 1, d_spr);
    g0w = d_spr;
  }
  k_spectral<<<gc, 128, 0, s>>>(d_K1, n, L, S, k->st, a, dt, k->Kt64, k->Kt32, k->trA, k->trRho,
                                g0w);
  VS_BUILD_TRY(cudaGetLastError());

  std::vector<float> host(nn);
  VS_BUILD_TRY(cudaMemcpyAsync(host.data(), k->Kt32, nn * sizeof(float), cudaMemcpyDeviceToHost, s));
  VS_BUILD_TRY(cudaStreamSynchronize(s));
  float kmax = 0.0f;
  bool finite = true;
  for (size_t i = 0; i < nn; ++i) {
    if (!isfinite(host[i])) finite = false;
    kmax = std::max(kmax, host[i]);
  }
  if (!finite) return fail(vs_set_error(VS_ERR_NONFINITE, "non-finite Green's function"));
  k->kmax = kmax;

  cudaFree(d_mlist);
  cudaFree(d_r);
  cudaFree(d_g);
  cudaFree(d_kper);
  cudaFree(d_T);
  cudaFree(d_K1);
  cudaFree(d_cos);
  cudaFree(d_spr);
  free_quad_rule(&q, s);
  cudaError_t e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    free_kernel_arrays(k);
    delete k;
    return vs_set_error(VS_ERR_CUDA, "make_kernel: %s", cudaGetErrorString(e));
  }
#undef VS_BUILD_TRY
  *out = k;
  return VS_OK;
}

extern "C" int vs_kernel_spectrum(vs_kernel k, double* out_host) {
  if (!k || !out_host) return vs_set_error(VS_ERR_INVALID_ARG, "NULL kernel or output");
  VS_CUDA_TRY(cudaMemcpy(out_host, k->Kt64, sizeof(double) * k->n * k->n, cudaMemcpyDeviceToHost));
  return VS_OK;
}

extern "C" int vs_kernel_radial(vs_kernel k, double* out_host, int* m_max_out) {
  if (!k || !m_max_out) return vs_set_error(VS_ERR_INVALID_ARG, "NULL kernel or m_max_out");
  *m_max_out = k->m_max;
  if (out_host)
    VS_CUDA_TRY(cudaMemcpy(out_host, k->radial, sizeof(double) * ((size_t)k->m_max + 1),
                           cudaMemcpyDeviceToHost));
  return VS_OK;
}
