// Declarations shared by the solver translation units: the per-map descriptor
// every solve kernel reads, the status flags of the fused update, a block
// reduction, and the host interface of the cluster engine (vs_cluster.cu).
#pragma once

#include <cuda_runtime.h>
#include <stddef.h>
#include <stdint.h>

#include "varsim.h"

namespace vsk {

constexpr int kFlagRunaway = 1;    // 1 - alpha s u fell below 0.05 somewhere
constexpr int kFlagNonfinite = 2;  // a non-finite temperature was produced

struct MapDesc {
  const float* p_dyn;
  const float* p_leak0;
  const float* s;
  float* theta;
  const float* theta_init;  // warm start (nullable)
  float* work;           // n*n, transposed spectral scratch
  const float* Kt;       // n*n cosine-basis kernel
  const float2* tw4n;
  const int* digrev;
  const float* trA;      // transient only
  const float* trRho;
  float* state;          // transient per-mode state, n*n
  float* work2;          // second scratch map (tensor-core path)
  const uint8_t* tcf;    // pre-tiled forward DCT matrix, BF16 hi/lo (tensor-core path)
  const uint8_t* tci;    // pre-tiled inverse DCT matrix
  float kmax;
  int n, rb, cb;
  int row_off, col_off, part_off;
};

// Convergence test of iterate `it` with update r (max |theta_n - theta_{n-1}|)
// and the previous update prev. VS_STOP_UPDATE: r <= tol. VS_STOP_ESTIMATE
// (from the second iterate on): the a-posteriori error estimate r q / (1 - q)
// <= tol, q = min(0.9, 4 r / prev) the contraction factor seen over the last
// two updates with a safety factor of 4.
__device__ __forceinline__ bool converged(float r, float prev, int it, float tol, int rule) {
  if (rule == VS_STOP_ESTIMATE && it > 1) {
    const float q = fminf(0.9f, 4.f * __fdividef(r, prev));
    return r * q <= tol * (1.f - q);
  }
  return r <= tol;
}

// Sum of one double per thread over the block (valid in thread 0).
__device__ __forceinline__ double block_sum(double v, double* red) {
  for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
  int w = threadIdx.x >> 5, l = threadIdx.x & 31;
  if (l == 0) red[w] = v;
  __syncthreads();
  double r = 0.0;
  if (threadIdx.x == 0)
    for (int i = 0; i < (int)(blockDim.x >> 5); ++i) r += red[i];
  __syncthreads();
  return r;  // valid in thread 0
}

// ---------------------------------------------------------------- cluster engine
constexpr int kClMaxN = 256;       // largest grid side the cluster engine takes
constexpr int kClMaxRanks = 8;     // CTAs per cluster at most

struct ClusterDev {
  const MapDesc* maps;
  const int* order;      // cluster index -> map index
  vs_solve_info* info;
  int max_iter;
  float beta, alpha, tol;
  int stop_rule;         // VS_STOP_*
  int cf_mode;           // closed-form instantiation: VS_CF_CONV or VS_CF_IMPULSE
  // physics-variant instantiation (beta above is then the preconditioner slope)
  int cond;              // VS_COND_*
  float one_me, t_amb;   // Kirchhoff: 1 - eta, T_amb
  int leak_n;            // 0 or the points of a piecewise-linear leakage factor
  float leak_x[VS_MAX_LEAK_POINTS], leak_y[VS_MAX_LEAK_POINTS];
};

// Launch shape of the cluster kernel for grid side n: CTAs per cluster,
// threads per CTA, dynamic shared memory per CTA.
struct ClHost {
  int ranks, threads;
  size_t smem;
};

using ClusterFn = void (*)(ClusterDev);

bool cluster_size_ok(int n);
ClHost cluster_shape(int n);
// The instantiation for n (32, 64, 128 or 256) and update-load batch (1, 2
// or 4; the default launch shape is 2).
ClusterFn cluster_kernel(int n, int batch);
// The instantiation with the physics variants in the update (batch 2).
ClusterFn cluster_kernel_phys(int n);
// The one-shot closed form on the cluster layout (n in [32, 256]), one
// cluster per map of P.maps / P.order, P.cf_mode the closed-form mode.
cudaError_t cluster_cf_launch(int n, const ClusterDev& P, int count, cudaStream_t s);
constexpr int kClBatches[3] = {1, 2, 4};
constexpr int kClBatchDefault = 2;

}  // namespace vsk
