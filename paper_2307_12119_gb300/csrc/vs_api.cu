// C ABI glue: error reporting, argument validation, version.
#include <math.h>
#include <stdarg.h>
#include <stdio.h>
#include <string.h>

#include "vs_internal.cuh"

namespace {
thread_local char g_err[1024] = "";
}

int vs_set_error(int status, const char* fmt, ...) {
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(g_err, sizeof(g_err), fmt, ap);
  va_end(ap);
  return status;
}

extern "C" const char* vs_last_error(void) { return g_err; }

extern "C" const char* vs_version(void) { return "varsim-gb300 0.1 (sm_103a)"; }

extern "C" const char* vs_status_string(int s) {
  switch (s) {
    case VS_OK: return "ok";
    case VS_ERR_INVALID_ARG: return "invalid argument";
    case VS_ERR_CUDA: return "CUDA error";
    case VS_ERR_OOM: return "out of device memory";
    case VS_ERR_NO_CONVERGENCE: return "no convergence";
    case VS_ERR_RUNAWAY: return "thermal or conductivity runaway";
    case VS_ERR_NONFINITE: return "non-finite value";
    case VS_ERR_TIMEOUT: return "grid barrier timed out";
    default: return "unknown status";
  }
}

static bool pos_finite(double v) { return isfinite(v) && v > 0.0; }

int vs_validate_stack(const vs_stack* s) {
  if (!s) return vs_set_error(VS_ERR_INVALID_ARG, "stack is NULL");
  if (s->n_layers < 1 || s->n_layers > VS_MAX_LAYERS)
    return vs_set_error(VS_ERR_INVALID_ARG, "n_layers %d outside [1, %d]", s->n_layers, VS_MAX_LAYERS);
  for (int i = 0; i < s->n_layers; ++i) {
    if (!pos_finite(s->thickness_m[i]) || !pos_finite(s->kappa_W_mK[i]))
      return vs_set_error(VS_ERR_INVALID_ARG, "layer %d: thickness and conductivity must be > 0", i);
  }
  if (!pos_finite(s->h_conv_W_m2K)) return vs_set_error(VS_ERR_INVALID_ARG, "h_conv must be > 0");
  if (!(s->heat_cap_J_m2K >= 0.0) || !isfinite(s->heat_cap_J_m2K))
    return vs_set_error(VS_ERR_INVALID_ARG, "heat_cap must be >= 0");
  if (s->spreader_layer != 0) {
    if (s->spreader_layer < 1 || s->spreader_layer >= s->n_layers)
      return vs_set_error(VS_ERR_INVALID_ARG, "spreader_layer %d outside [1, %d)",
                          s->spreader_layer, s->n_layers);
    if (!pos_finite(s->spreader_side_m))
      return vs_set_error(VS_ERR_INVALID_ARG, "spreader_side_m must be > 0");
  }
  return VS_OK;
}

int vs_validate_grid(const vs_grid* g) {
  if (!g) return vs_set_error(VS_ERR_INVALID_ARG, "grid is NULL");
  if (g->n < VS_MIN_N || g->n > VS_MAX_N || (g->n & (g->n - 1)))
    return vs_set_error(VS_ERR_INVALID_ARG, "n = %d must be a power of two in [%d, %d]", g->n,
                        VS_MIN_N, VS_MAX_N);
  if (!pos_finite(g->die_m)) return vs_set_error(VS_ERR_INVALID_ARG, "die size must be > 0");
  return VS_OK;
}

int vs_validate_params(const vs_solve_params* p) {
  if (!p) return vs_set_error(VS_ERR_INVALID_ARG, "params is NULL");
  if (!(p->beta_per_K >= 0.0) || !isfinite(p->beta_per_K))
    return vs_set_error(VS_ERR_INVALID_ARG, "beta must be finite and >= 0");
  if (!(p->alpha_per_K >= 0.0) || !isfinite(p->alpha_per_K))
    return vs_set_error(VS_ERR_INVALID_ARG, "alpha must be finite and >= 0");
  if (!pos_finite(p->tol_K)) return vs_set_error(VS_ERR_INVALID_ARG, "tol must be > 0");
  if (p->max_iter < 1 || p->max_iter > 1000)
    return vs_set_error(VS_ERR_INVALID_ARG, "max_iter %d outside [1, 1000]", p->max_iter);
  if (p->precision != VS_PREC_FP32 && p->precision != VS_PREC_BF16_SPLIT)
    return vs_set_error(VS_ERR_INVALID_ARG, "unknown precision %d", p->precision);
  if (p->engine != VS_ENGINE_AUTO && p->engine != VS_ENGINE_STREAMED &&
      p->engine != VS_ENGINE_CLUSTER)
    return vs_set_error(VS_ERR_INVALID_ARG, "unknown engine %d", p->engine);
  if (p->stop_rule != VS_STOP_UPDATE && p->stop_rule != VS_STOP_ESTIMATE)
    return vs_set_error(VS_ERR_INVALID_ARG, "unknown stopping rule %d", p->stop_rule);
  if (p->conductivity != VS_COND_LINEAR && p->conductivity != VS_COND_KIRCHHOFF)
    return vs_set_error(VS_ERR_INVALID_ARG, "unknown conductivity model %d", p->conductivity);
  if (p->conductivity == VS_COND_KIRCHHOFF &&
      (!pos_finite(p->eta) || fabs(p->eta - 1.0) < 1e-6 || !pos_finite(p->t_amb_K)))
    return vs_set_error(VS_ERR_INVALID_ARG, "Kirchhoff model needs eta > 0, eta != 1 and T_amb > 0");
  if (p->leak_points != 0) {
    if (p->leak_points < 2 || p->leak_points > VS_MAX_LEAK_POINTS)
      return vs_set_error(VS_ERR_INVALID_ARG, "leak_points %d not 0 or in [2, %d]", p->leak_points,
                          VS_MAX_LEAK_POINTS);
    for (int i = 0; i < p->leak_points; ++i) {
      if (!isfinite(p->leak_theta_K[i]) || !isfinite(p->leak_g[i]))
        return vs_set_error(VS_ERR_INVALID_ARG, "leakage table entry %d is not finite", i);
      if (i && !(p->leak_theta_K[i] > p->leak_theta_K[i - 1]))
        return vs_set_error(VS_ERR_INVALID_ARG, "leakage table temperatures must increase");
    }
  }
  return VS_OK;
}

int vs_params_physics(const vs_solve_params* p) {
  return p->conductivity != VS_COND_LINEAR || p->leak_points != 0;
}

void vs_stack_to_dev(const vs_stack* s, vs_stack_dev* d) {
  memset(d, 0, sizeof(*d));
  d->n_layers = s->n_layers;
  for (int i = 0; i < s->n_layers; ++i) {
    d->t[i] = s->thickness_m[i];
    d->kappa[i] = s->kappa_W_mK[i];
  }
  d->h = s->h_conv_W_m2K;
  d->heat_cap = s->heat_cap_J_m2K;
  d->spreader_layer = s->spreader_layer;
  d->spreader_side = s->spreader_side_m;
}
