// Internal declarations shared by the translation units of libvarsim.
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>

#include "varsim.h"

// ---------------------------------------------------------------- errors

int vs_set_error(int status, const char* fmt, ...);

#define VS_CUDA_TRY(call)                                                    \
  do {                                                                        \
    cudaError_t e_ = (call);                                                  \
    if (e_ != cudaSuccess) {                                                  \
      return vs_set_error(e_ == cudaErrorMemoryAllocation ? VS_ERR_OOM        \
                                                          : VS_ERR_CUDA,      \
                          "%s failed: %s (%s:%d)", #call,                     \
                          cudaGetErrorString(e_), __FILE__, __LINE__);        \
    }                                                                         \
  } while (0)

// ---------------------------------------------------------------- stack

struct vs_stack_dev {
  int n_layers;
  double t[VS_MAX_LAYERS];
  double kappa[VS_MAX_LAYERS];
  double h;
  double heat_cap;
  int spreader_layer;      // 0: die-sized stack
  double spreader_side;    // metres, >= the die side when spreader_layer > 0
};

// ---------------------------------------------------------------- FFT tables
// Per grid size n: twiddles W_{4n}^e = exp(-2 pi i e / (4n)), e in [0, 4n)
// (float2), and the digit-reversal map of the in-place radix-16/8/4/2 FFT.
struct vs_fft_tables {
  int n;
  float2* tw4n;      // device [4n]
  int* digrev;       // device [n]
};

const vs_fft_tables* vs_get_fft_tables(int n, int* status);

// ---------------------------------------------------------------- kernel
struct vs_kernel_t {
  int n;
  double die_m;
  vs_stack_dev st;
  int quad_nodes;
  double rel_tol;
  double* Kt64;        // device [n][n] FP64 cosine-basis kernel
  float* Kt32;         // device [n][n]
  float kmax;          // max over modes of K (host)
  double* radial;      // device [m_max + 1] top-layer radial table
  int m_max;
  double dt;           // transient step (0 = none)
  float* trA;          // device [n][n] primary-mode weight cell^-2 g D
  float* trRho;        // device [n][n] exp(-dt / (C g))
  const vs_fft_tables* fft;
};

int vs_validate_stack(const vs_stack* s);
int vs_validate_grid(const vs_grid* g);
int vs_validate_params(const vs_solve_params* p);
// Non-zero if the parameters ask for a physics variant (Kirchhoff conductivity
// or piecewise-linear leakage), which only the streamed engine runs.
int vs_params_physics(const vs_solve_params* p);
void vs_stack_to_dev(const vs_stack* s, vs_stack_dev* d);

// Hankel quadrature of the top-layer radial Green's function at `count`
// radii (device arrays), see vs_kernel_build.cu.
int vs_hankel_eval(const vs_stack_dev& st, double cell_m, int quad_nodes,
                   const double* r_dev, double* out_dev, int count, cudaStream_t s);

// ---------------------------------------------------------------- tensor-core cluster engine
// BF16 hi/lo split engine with the map on chip (vs_tcc.cu): n = 256, cold
// starts, linear models. vs_tcc_launch runs `count` maps (cluster index ->
// map through P.order).
namespace vsk { struct ClusterDev; }
bool vs_tcc_ok(int n);
int vs_tcc_check(cudaStream_t s);
int vs_tcc_launch(const vsk::ClusterDev& P, int count, cudaStream_t s);

// ---------------------------------------------------------------- network
// 3x3 convolution of the warm-start network as a tcgen05 implicit GEMM
// (vs_conv_tc.cu; BF16 activations and weights, FP32 accumulation), for
// inference. W: the layer's BF16 weights [cout][cin][3][3]. Returns VS_OK, an
// error, or -1 if the layer's shape does not fit the kernel.
int vs_conv_tc(const float* in, int in_ctot, int cin, const void* W, const float* bias,
               float* out, int out_ctot, int cout, int B, int H, int relu, cudaStream_t s);

// ---------------------------------------------------------------- transient
// Persistent transient of one map (vs_transient.cu): lagged leakage,
// untruncated superposition, n in {256, 512, 1024}. Returns the map's status
// (info filled), an error, or -1 if the launch shape does not fit the device.
bool vs_transient_fast_ok(int n);
int vs_transient_fast(vs_kernel k, int n_steps, const float* p_dyn_trace, const float* p_leak0,
                      const float* s_kappa, const vs_solve_params* params, int implicit,
                      int window, float* theta_trace, vs_solve_info* info, cudaStream_t s);

// ---------------------------------------------------------------- plans
// Asynchronous copy of a plan's per-map outcome to (pinned) host memory.
int vs_plan_info_async(vs_plan p, vs_solve_info* info_host, cudaStream_t s);
// VS_ERR_TIMEOUT if the plan's last run aborted on a barrier timeout (syncs s).
int vs_plan_check_timeout(vs_plan p, cudaStream_t s);
