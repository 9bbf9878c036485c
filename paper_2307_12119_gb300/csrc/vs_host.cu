// Batched steady solve from and to host memory: the maps are streamed through
// the GPU in chunks, with the host-to-device copies of chunk i+1 and the
// device-to-host copy of chunk i-1 overlapped with the solve of chunk i
// (three streams, two device buffer slots, events between them). The solve of
// a chunk is the plan of vs_plan_create over that chunk, so every map gets
// exactly the result vs_solve_batch gives it.
#include <string.h>

#include <algorithm>
#include <vector>

#include "vs_internal.cuh"

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

struct Job {
  Slot slot[2];
  cudaStream_t h2d = nullptr, comp = nullptr, d2h = nullptr;
  cudaEvent_t start = nullptr;
  vs_solve_info* stage = nullptr;   // pinned per-map outcomes

  ~Job() {
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

int make_plan(vs_kernel k, const Slot& s, int maps, const vs_solve_params* prm, vs_plan* out,
              cudaStream_t st) {
  const size_t nn = (size_t)k->n * k->n;
  std::vector<vs_batch_item> items(maps);
  for (int i = 0; i < maps; ++i)
    items[i] = vs_batch_item{k, s.pd + i * nn, s.pl + i * nn, s.sk ? s.sk + i * nn : nullptr,
                             s.th + i * nn, nullptr};
  return vs_plan_create(items.data(), maps, prm, out, st);
}

}  // namespace

extern "C" int vs_solve_batch_host(vs_kernel k, int count, const float* p_dyn, const float* p_leak0,
                                   const float* s_kappa, float* theta,
                                   const vs_solve_params* params, vs_solve_info* info_host,
                                   int chunk_maps, void* stream) {
  if (!k) return vs_set_error(VS_ERR_INVALID_ARG, "NULL kernel");
  if (count < 1) return vs_set_error(VS_ERR_INVALID_ARG, "count %d < 1", count);
  if (!p_dyn || !p_leak0 || !theta) return vs_set_error(VS_ERR_INVALID_ARG, "NULL map");
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
  const int nchunks = (count + chunk - 1) / chunk;
  const int nslots = std::min(2, nchunks);
  const int tail = count - (nchunks - 1) * chunk;

  Job job;
  VS_CUDA_TRY(cudaStreamCreateWithFlags(&job.h2d, cudaStreamNonBlocking));
  VS_CUDA_TRY(cudaStreamCreateWithFlags(&job.comp, cudaStreamNonBlocking));
  VS_CUDA_TRY(cudaStreamCreateWithFlags(&job.d2h, cudaStreamNonBlocking));
  VS_CUDA_TRY(cudaEventCreateWithFlags(&job.start, cudaEventDisableTiming));
  VS_CUDA_TRY(cudaMallocHost(&job.stage, sizeof(vs_solve_info) * count));
  for (int si = 0; si < nslots; ++si) {
    Slot& s = job.slot[si];
    VS_CUDA_TRY(cudaMalloc(&s.pd, chunk * mb));
    VS_CUDA_TRY(cudaMalloc(&s.pl, chunk * mb));
    if (s_kappa) VS_CUDA_TRY(cudaMalloc(&s.sk, chunk * mb));
    VS_CUDA_TRY(cudaMalloc(&s.th, chunk * mb));
    VS_CUDA_TRY(cudaEventCreateWithFlags(&s.in_ready, cudaEventDisableTiming));
    VS_CUDA_TRY(cudaEventCreateWithFlags(&s.done, cudaEventDisableTiming));
    VS_CUDA_TRY(cudaEventCreateWithFlags(&s.out_done, cudaEventDisableTiming));
    rc = make_plan(k, s, chunk, params, &s.full, job.comp);
    if (rc) return rc;
    // the last chunk is solved in slot (nchunks - 1) % nslots
    if (tail != chunk && si == (nchunks - 1) % nslots) {
      rc = make_plan(k, s, tail, params, &s.tail, job.comp);
      if (rc) return rc;
    }
  }
  // everything queued on `stream` before this call comes first
  VS_CUDA_TRY(cudaEventRecord(job.start, (cudaStream_t)stream));
  VS_CUDA_TRY(cudaStreamWaitEvent(job.h2d, job.start, 0));
  VS_CUDA_TRY(cudaStreamWaitEvent(job.comp, job.start, 0));
  VS_CUDA_TRY(cudaStreamWaitEvent(job.d2h, job.start, 0));

  for (int i = 0; i < nchunks; ++i) {
    Slot& s = job.slot[i % nslots];
    const size_t off = (size_t)i * chunk * nn;
    const int m = std::min(chunk, count - i * chunk);
    const size_t bytes = (size_t)m * mb;
    // inputs of this slot are free once the solve of chunk i - nslots is done
    // (one copy stream: more streams do not raise the host link's rate)
    if (i >= nslots) VS_CUDA_TRY(cudaStreamWaitEvent(job.h2d, s.done, 0));
    VS_CUDA_TRY(cudaMemcpyAsync(s.pd, p_dyn + off, bytes, cudaMemcpyHostToDevice, job.h2d));
    VS_CUDA_TRY(cudaMemcpyAsync(s.pl, p_leak0 + off, bytes, cudaMemcpyHostToDevice, job.h2d));
    if (s_kappa)
      VS_CUDA_TRY(cudaMemcpyAsync(s.sk, s_kappa + off, bytes, cudaMemcpyHostToDevice, job.h2d));
    VS_CUDA_TRY(cudaEventRecord(s.in_ready, job.h2d));
    // the solve also needs the slot's theta free (copied out for chunk i - nslots)
    VS_CUDA_TRY(cudaStreamWaitEvent(job.comp, s.in_ready, 0));
    if (i >= nslots) VS_CUDA_TRY(cudaStreamWaitEvent(job.comp, s.out_done, 0));
    vs_plan plan = (m == chunk) ? s.full : s.tail;
    rc = vs_plan_run(plan, job.comp);
    if (rc) return rc;
    VS_CUDA_TRY(cudaEventRecord(s.done, job.comp));
    VS_CUDA_TRY(cudaStreamWaitEvent(job.d2h, s.done, 0));
    VS_CUDA_TRY(cudaMemcpyAsync(theta + off, s.th, bytes, cudaMemcpyDeviceToHost, job.d2h));
    rc = vs_plan_info_async(plan, job.stage + (size_t)i * chunk, job.d2h);
    if (rc) return rc;
    VS_CUDA_TRY(cudaEventRecord(s.out_done, job.d2h));
  }
  VS_CUDA_TRY(cudaStreamSynchronize(job.h2d));
  VS_CUDA_TRY(cudaStreamSynchronize(job.comp));
  VS_CUDA_TRY(cudaStreamSynchronize(job.d2h));
  int worst = VS_OK;
  for (int si = 0; si < nslots; ++si) {
    for (vs_plan p : {job.slot[si].full, job.slot[si].tail}) {
      if (!p) continue;
      rc = vs_plan_check_timeout(p, job.comp);
      if (rc) return rc;
    }
  }
  for (int i = 0; i < count; ++i) worst = std::max(worst, job.stage[i].status);
  if (info_host) memcpy(info_host, job.stage, sizeof(vs_solve_info) * count);
  return worst;
}
