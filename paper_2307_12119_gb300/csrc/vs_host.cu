// Batched steady solve from and to host memory: the maps are streamed through
// the GPU in chunks, with the host-to-device copies of chunk i+1 and the
// device-to-host copy of chunk i-1 overlapped with the solve of chunk i
// (three streams, two device buffer slots, events between them). The solve of
// a chunk is a plan over that chunk's device buffers, so every map gets
// exactly the result vs_solve_batch gives it. A host plan keeps the streams,
// buffers and chunk plans for repeated runs; vs_solve_batch_host makes one
// per call.
#include <string.h>

#include <algorithm>
#include <vector>

#include "vs_internal.cuh"

int plan_create(const vs_batch_item* items_host, int n_items, const vs_solve_params* params,
                int shape, vs_plan* out, void* stream);

namespace {

struct Slot {
  float* pd = nullptr;
  float* pl = nullptr;
  float* sk = nullptr;
  float* th = nullptr;
  vs_plan full = nullptr;      // plan over `chunk` maps
  vs_plan tail = nullptr;      // plan over the last, shorter chunk (if any)
  cudaEvent_t in_ready = nullptr, done = nullptr, out_done = nullptr;
};

int make_plan(vs_kernel k, const Slot& s, int maps, const vs_solve_params* prm, vs_plan* out,
              cudaStream_t st) {
  const size_t nn = (size_t)k->n * k->n;
  std::vector<vs_batch_item> items(maps);
  for (int i = 0; i < maps; ++i)
    items[i] = vs_batch_item{k, s.pd + i * nn, s.pl + i * nn, s.sk ? s.sk + i * nn : nullptr,
                             s.th + i * nn, nullptr};
  // the buffers do not hold maps yet: the cached launch shape or the default,
  // no timing runs
  return plan_create(items.data(), maps, prm, -1, out, st);
}

}  // namespace

struct vs_host_plan_t {
  vs_kernel k = nullptr;
  int count = 0, chunk = 0, nchunks = 0, nslots = 0, with_s = 0;
  Slot slot[2];
  cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
  cudaEvent_t start = nullptr;
  vs_solve_info* stage = nullptr;   // pinned per-map outcomes

  ~vs_host_plan_t() {
    for (Slot& s : slot) {
      vs_plan_free(s.full);
      vs_plan_free(s.tail);
      cudaFree(s.pd);
      cudaFree(s.pl);
      cudaFree(s.sk);
      cudaFree(s.th);
      if (s.in_ready) cudaEventDestroy(s.in_ready);
      if (s.done) cudaEventDestroy(s.done);
      if (s.out_done) cudaEventDestroy(s.out_done);
    }
    if (start) cudaEventDestroy(start);
    if (h2d) cudaStreamDestroy(h2d);
    if (comp) cudaStreamDestroy(comp);
    if (d2h) cudaStreamDestroy(d2h);
    cudaFreeHost(stage);
  }
};

extern "C" int vs_host_plan_create(vs_kernel k, int count, int with_s, const vs_solve_params* params,
                                   int chunk_maps, vs_host_plan* out) {
  if (!out) return vs_set_error(VS_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!k) return vs_set_error(VS_ERR_INVALID_ARG, "NULL kernel");
  if (count < 1) return vs_set_error(VS_ERR_INVALID_ARG, "count %d < 1", count);
  if (chunk_maps < 0) return vs_set_error(VS_ERR_INVALID_ARG, "chunk_maps %d < 0", chunk_maps);
  int rc = vs_validate_params(params);
  if (rc) return rc;
  const size_t nn = (size_t)k->n * k->n, mb = nn * sizeof(float);
  // default: a sixteenth of the batch (short pipeline fill and drain), at
  // most about 1 GiB of device buffers per slot
  int chunk = chunk_maps > 0 ? chunk_maps
                             : (int)std::max<size_t>(1, std::min<size_t>((count + 15) / 16,
                                                                          ((size_t)1 << 30) / (4 * mb)));
  chunk = std::min(chunk, count);
  vs_host_plan_t* hp = new vs_host_plan_t;
  hp->k = k;
  hp->count = count;
  hp->chunk = chunk;
  hp->nchunks = (count + chunk - 1) / chunk;
  hp->nslots = std::min(2, hp->nchunks);
  hp->with_s = with_s ? 1 : 0;
  const int tail = count - (hp->nchunks - 1) * chunk;
  auto fail = [&](int code) {
    delete hp;
    return code;
  };
#define HP_TRY(x)                                                                          \
  do {                                                                                     \
    cudaError_t e_ = (x);                                                                  \
    if (e_ != cudaSuccess)                                                                 \
      return fail(vs_set_error(e_ == cudaErrorMemoryAllocation ? VS_ERR_OOM : VS_ERR_CUDA, \
                               "%s: %s", #x, cudaGetErrorString(e_)));                     \
  } while (0)
  HP_TRY(cudaStreamCreateWithFlags(&hp->h2d, cudaStreamNonBlocking));
  HP_TRY(cudaStreamCreateWithFlags(&hp->comp, cudaStreamNonBlocking));
  HP_TRY(cudaStreamCreateWithFlags(&hp->d2h, cudaStreamNonBlocking));
  HP_TRY(cudaEventCreateWithFlags(&hp->start, cudaEventDisableTiming));
  HP_TRY(cudaMallocHost(&hp->stage, sizeof(vs_solve_info) * count));
  for (int si = 0; si < hp->nslots; ++si) {
    Slot& s = hp->slot[si];
    HP_TRY(cudaMalloc(&s.pd, chunk * mb));
    HP_TRY(cudaMalloc(&s.pl, chunk * mb));
    if (hp->with_s) HP_TRY(cudaMalloc(&s.sk, chunk * mb));
    HP_TRY(cudaMalloc(&s.th, chunk * mb));
    HP_TRY(cudaEventCreateWithFlags(&s.in_ready, cudaEventDisableTiming));
    HP_TRY(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
    HP_TRY(cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming));
    rc = make_plan(k, s, chunk, params, &s.full, hp->comp);
    if (rc) return fail(rc);
    // the last chunk is solved in slot (nchunks - 1) % nslots
    if (tail != chunk && si == (hp->nchunks - 1) % hp->nslots) {
      rc = make_plan(k, s, tail, params, &s.tail, hp->comp);
      if (rc) return fail(rc);
    }
  }
#undef HP_TRY
  *out = hp;
  return VS_OK;
}

extern "C" int vs_host_plan_run(vs_host_plan hp, const float* p_dyn, const float* p_leak0,
                                const float* s_kappa, float* theta, vs_solve_info* info_host,
                                void* stream) {
  if (!hp) return vs_set_error(VS_ERR_INVALID_ARG, "NULL host plan");
  if (!p_dyn || !p_leak0 || !theta) return vs_set_error(VS_ERR_INVALID_ARG, "NULL map");
  if ((s_kappa != nullptr) != (hp->with_s != 0))
    return vs_set_error(VS_ERR_INVALID_ARG, "s_kappa must be given exactly when the host plan was "
                                            "created with with_s = 1");
  const size_t nn = (size_t)hp->k->n * hp->k->n, mb = nn * sizeof(float);
  const int chunk = hp->chunk, nslots = hp->nslots, count = hp->count;
  // everything queued on `stream` before this call comes first
  VS_CUDA_TRY(cudaEventRecord(hp->start, (cudaStream_t)stream));
  VS_CUDA_TRY(cudaStreamWaitEvent(hp->h2d, hp->start, 0));
  VS_CUDA_TRY(cudaStreamWaitEvent(hp->comp, hp->start, 0));
  VS_CUDA_TRY(cudaStreamWaitEvent(hp->d2h, hp->start, 0));
  int rc = VS_OK;
  for (int i = 0; i < hp->nchunks; ++i) {
    Slot& s = hp->slot[i % nslots];
    const size_t off = (size_t)i * chunk * nn;
    const int m = std::min(chunk, count - i * chunk);
    const size_t bytes = (size_t)m * mb;
    // inputs of this slot are free once the solve of chunk i - nslots is done
    // (one copy stream: more streams do not raise the host link's rate)
    if (i >= nslots) VS_CUDA_TRY(cudaStreamWaitEvent(hp->h2d, s.done, 0));
    VS_CUDA_TRY(cudaMemcpyAsync(s.pd, p_dyn + off, bytes, cudaMemcpyHostToDevice, hp->h2d));
    VS_CUDA_TRY(cudaMemcpyAsync(s.pl, p_leak0 + off, bytes, cudaMemcpyHostToDevice, hp->h2d));
    if (s_kappa)
      VS_CUDA_TRY(cudaMemcpyAsync(s.sk, s_kappa + off, bytes, cudaMemcpyHostToDevice, hp->h2d));
    VS_CUDA_TRY(cudaEventRecord(s.in_ready, hp->h2d));
    // the solve also needs the slot's theta free (copied out for chunk i - nslots)
    VS_CUDA_TRY(cudaStreamWaitEvent(hp->comp, s.in_ready, 0));
    if (i >= nslots) VS_CUDA_TRY(cudaStreamWaitEvent(hp->comp, s.out_done, 0));
    vs_plan plan = (m == chunk) ? s.full : s.tail;
    rc = vs_plan_run(plan, hp->comp);
    if (rc) return rc;
    VS_CUDA_TRY(cudaEventRecord(s.done, hp->comp));
    VS_CUDA_TRY(cudaStreamWaitEvent(hp->d2h, s.done, 0));
    VS_CUDA_TRY(cudaMemcpyAsync(theta + off, s.th, bytes, cudaMemcpyDeviceToHost, hp->d2h));
    rc = vs_plan_info_async(plan, hp->stage + (size_t)i * chunk, hp->d2h);
    if (rc) return rc;
    VS_CUDA_TRY(cudaEventRecord(s.out_done, hp->d2h));
  }
  VS_CUDA_TRY(cudaStreamSynchronize(hp->h2d));
  VS_CUDA_TRY(cudaStreamSynchronize(hp->comp));
  VS_CUDA_TRY(cudaStreamSynchronize(hp->d2h));
  for (int si = 0; si < nslots; ++si) {
    for (vs_plan p : {hp->slot[si].full, hp->slot[si].tail}) {
      if (!p) continue;
      rc = vs_plan_check_timeout(p, hp->comp);
      if (rc) return rc;
    }
  }
  int worst = VS_OK;
  for (int i = 0; i < count; ++i) worst = std::max(worst, hp->stage[i].status);
  if (info_host) memcpy(info_host, hp->stage, sizeof(vs_solve_info) * count);
  return worst;
}

extern "C" void vs_host_plan_free(vs_host_plan hp) { delete hp; }

extern "C" int vs_solve_batch_host(vs_kernel k, int count, const float* p_dyn, const float* p_leak0,
                                   const float* s_kappa, float* theta,
                                   const vs_solve_params* params, vs_solve_info* info_host,
                                   int chunk_maps, void* stream) {
  if (!k) return vs_set_error(VS_ERR_INVALID_ARG, "NULL kernel");
  if (!p_dyn || !p_leak0 || !theta) return vs_set_error(VS_ERR_INVALID_ARG, "NULL map");
  vs_host_plan hp = nullptr;
  int rc = vs_host_plan_create(k, count, s_kappa != nullptr, params, chunk_maps, &hp);
  if (rc) return rc;
  rc = vs_host_plan_run(hp, p_dyn, p_leak0, s_kappa, theta, info_host, stream);
  vs_host_plan_free(hp);
  return rc;
}
