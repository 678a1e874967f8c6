// Several grids per call (sph_filter_batch_*), CUDA-graph capture of the per-substep filter
// applications, and the per-plan autotuner of the staged shell kernel's launch shape.
#include <algorithm>
#include <vector>

#include "internal.h"

struct sph_filter_batch_s {
  int device = 0;
  std::vector<sph_filter_plan_s*> plans;
  std::vector<cudaStream_t> streams;  // one per grid
  std::vector<cudaEvent_t> joins;     // one per grid
  cudaEvent_t fork = nullptr;
  cudaStream_t cap = nullptr;         // capture stream
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  sph::TcBatch* tcb = nullptr;        // every plan in the tensor-core form: one launch for all grids
};

namespace {

void drop_graph(sph_filter_batch_s* b) {
  if (b->exec) cudaGraphExecDestroy(b->exec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->exec = nullptr;
  b->graph = nullptr;
}

void free_batch(sph_filter_batch_s* b) {
  if (!b) return;
  drop_graph(b);
  sph::tc_batch_free(b->tcb);
  for (cudaStream_t s : b->streams) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->joins) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  if (b->cap) cudaStreamDestroy(b->cap);
  delete b;
}

// Filter every grid: one persistent launch over all grids for tensor-core plans; otherwise fork from
// `s` to the per-grid streams, launch each plan and join back into `s`.
sph_status enqueue(sph_filter_batch_s* b, const double* const* in, double* const* out, cudaStream_t s) {
  if (b->tcb) {
    int cur = -1;
    cudaGetDevice(&cur);
    if (cur != b->device) cudaSetDevice(b->device);
    const cudaError_t e = sph::tc_batch_launch(b->tcb, in, out, s);
    if (cur != b->device) cudaSetDevice(cur);
    return e == cudaSuccess ? SPH_OK : SPH_ECUDA;
  }
  if (cudaEventRecord(b->fork, s) != cudaSuccess) return SPH_ECUDA;
  for (size_t g = 0; g < b->plans.size(); ++g) {
    if (cudaStreamWaitEvent(b->streams[g], b->fork, 0) != cudaSuccess) return SPH_ECUDA;
    const sph_status st =
        sph::launch_plan(b->plans[g], in[g], nullptr, out[g], sph::kMapNone, sph::kOutNone, 0, 0, b->streams[g]);
    if (st != SPH_OK) return st;
    if (cudaEventRecord(b->joins[g], b->streams[g]) != cudaSuccess) return SPH_ECUDA;
  }
  for (size_t g = 0; g < b->plans.size(); ++g)
    if (cudaStreamWaitEvent(s, b->joins[g], 0) != cudaSuccess) return SPH_ECUDA;
  return SPH_OK;
}

struct Shape {
  int threads, batch_th, batch_ph;
  size_t smem;
};

// Launch shapes of the staged kernel that fit the device: threads per CTA and sequences per FFT batch.
std::vector<Shape> candidates(sph_filter_plan_s* p) {
  std::vector<Shape> out;
  if (p->cluster) {  // the cluster kernel's batches are set by the free buffer memory
    out.push_back(Shape{p->threads2, p->args2.batch_th, p->args2.batch_ph, p->smem2});
    return out;
  }
  const size_t optin = (size_t)sph::max_smem_optin(p->device);
  sph::ShellArgs2 a = p->args2;
  const int nseq = (p->Nph / 2 + 1) / 2;
  const int npair = (p->Nth + 1) / 2;
  const int thr[2] = {256, 512};
  for (int ti = 0; ti < 2; ++ti) {
    for (int div = 1; div <= 64; div *= 2) {
      a.batch_th = std::max(1, (nseq + div - 1) / div);
      a.batch_ph = std::max(1, (npair + div - 1) / div);
      const size_t smem = sph::shell_smem_bytes(a, p->precision);
      if (smem <= optin) {
        bool dup = false;
        for (const Shape& s : out) dup |= s.threads == thr[ti] && s.batch_th == a.batch_th && s.batch_ph == a.batch_ph;
        if (!dup) out.push_back(Shape{thr[ti], a.batch_th, a.batch_ph, smem});
      }
      if (a.batch_th == 1 && a.batch_ph == 1) break;
    }
  }
  return out;
}

}  // namespace

extern "C" {

sph_status sph_filter_batch_create(sph_filter_batch* out, int nplans, const sph_filter_plan* plans) {
  if (!out) return SPH_EINVAL;
  *out = nullptr;
  if (nplans < 1 || !plans) return SPH_EINVAL;
  for (int g = 0; g < nplans; ++g)
    if (!plans[g] || plans[g]->device != plans[0]->device) return SPH_EINVAL;
  sph_filter_batch_s* b = new (std::nothrow) sph_filter_batch_s();
  if (!b) return SPH_ENOMEM;
  b->device = plans[0]->device;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(b->device);
  bool ok = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess &&
            cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking) == cudaSuccess;
  for (int g = 0; ok && g < nplans; ++g) {
    cudaStream_t s = nullptr;
    cudaEvent_t e = nullptr;
    ok = cudaStreamCreateWithFlags(&s, cudaStreamNonBlocking) == cudaSuccess &&
         cudaEventCreateWithFlags(&e, cudaEventDisableTiming) == cudaSuccess;
    if (s) b->streams.push_back(s);
    if (e) b->joins.push_back(e);
    b->plans.push_back(plans[g]);
  }
  bool all_tc = true;
  for (int g = 0; g < nplans; ++g) all_tc &= plans[g]->tc != nullptr;
  if (ok && all_tc) {
    const sph_status st = sph::tc_batch_setup(&b->tcb, b->plans.data(), nplans);
    if (st != SPH_OK && st != SPH_EUNSUPPORTED) ok = false;  // unsupported: per-grid launches instead
  }
  if (cur >= 0) cudaSetDevice(cur);
  if (!ok) {
    free_batch(b);
    return SPH_ECUDA;
  }
  *out = b;
  return SPH_OK;
}

void sph_filter_batch_destroy(sph_filter_batch batch) {
  if (!batch) return;
  int cur = -1;
  cudaGetDevice(&cur);
  cudaSetDevice(batch->device);
  cudaDeviceSynchronize();
  free_batch(batch);
  if (cur >= 0) cudaSetDevice(cur);
}

sph_status sph_filter_batch_apply(sph_filter_batch batch, const double* const* in, double* const* out,
                                  sph_stream_t stream) {
  if (!batch || !in || !out) return SPH_EINVAL;
  return enqueue(batch, in, out, (cudaStream_t)stream);
}

sph_status sph_filter_batch_capture(sph_filter_batch batch, const double* const* in, double* const* out, int napply,
                                    sph_stream_t stream) {
  if (!batch || !in || !out || napply < 1) return SPH_EINVAL;
  drop_graph(batch);
  // the capture stream first waits for work already queued on the caller's stream
  cudaEvent_t ready = nullptr;
  if (cudaEventCreateWithFlags(&ready, cudaEventDisableTiming) != cudaSuccess) return SPH_ECUDA;
  cudaEventRecord(ready, (cudaStream_t)stream);
  cudaStreamWaitEvent(batch->cap, ready, 0);
  cudaEventDestroy(ready);
  if (cudaStreamBeginCapture(batch->cap, cudaStreamCaptureModeThreadLocal) != cudaSuccess) return SPH_ECUDA;
  sph_status st = SPH_OK;
  for (int k = 0; k < napply && st == SPH_OK; ++k) st = enqueue(batch, k == 0 ? in : out, out, batch->cap);
  cudaGraph_t g = nullptr;
  const cudaError_t e = cudaStreamEndCapture(batch->cap, &g);
  if (st != SPH_OK || e != cudaSuccess) {
    if (g) cudaGraphDestroy(g);
    return st != SPH_OK ? st : SPH_ECUDA;
  }
  batch->graph = g;
  if (cudaGraphInstantiate(&batch->exec, g, 0) != cudaSuccess) {
    drop_graph(batch);
    return SPH_ECUDA;
  }
  return SPH_OK;
}

sph_status sph_filter_batch_launch(sph_filter_batch batch, sph_stream_t stream) {
  if (!batch || !batch->exec) return SPH_EINVAL;
  return cudaGraphLaunch(batch->exec, (cudaStream_t)stream) == cudaSuccess ? SPH_OK : SPH_ECUDA;
}

sph_status sph_filter_plan_autotune(sph_filter_plan plan, const double* in, double* out, sph_stream_t stream,
                                    double* best_ms) {
  if (!plan || !in || !out) return SPH_EINVAL;
  cudaStream_t s = (cudaStream_t)stream;
  cudaEvent_t e0 = nullptr, e1 = nullptr;
  if (cudaEventCreate(&e0) != cudaSuccess || cudaEventCreate(&e1) != cudaSuccess) return SPH_ECUDA;
  auto time_one = [&](float* ms) -> sph_status {
    sph_status st = sph::launch_plan(plan, in, nullptr, out, sph::kMapNone, sph::kOutNone, 0, 0, s);
    if (st != SPH_OK) return st;
    cudaEventRecord(e0, s);
    for (int k = 0; k < 3 && st == SPH_OK; ++k)
      st = sph::launch_plan(plan, in, nullptr, out, sph::kMapNone, sph::kOutNone, 0, 0, s);
    cudaEventRecord(e1, s);
    if (cudaEventSynchronize(e1) != cudaSuccess) return SPH_ECUDA;
    cudaEventElapsedTime(ms, e0, e1);
    *ms /= 3.0f;
    return st;
  };
  sph_status st = SPH_OK;
  float best = 0.0f;
  if (!plan->use_v2) {
    st = time_one(&best);
  } else {
    const std::vector<Shape> cand = candidates(plan);
    Shape keep{plan->threads2, plan->args2.batch_th, plan->args2.batch_ph, plan->smem2};
    best = -1.0f;
    for (const Shape& c : cand) {
      plan->threads2 = c.threads;
      plan->args2.batch_th = c.batch_th;
      plan->args2.batch_ph = c.batch_ph;
      plan->smem2 = c.smem;
      float ms = 0.0f;
      st = time_one(&ms);
      if (st != SPH_OK) break;
      if (best < 0.0f || ms < best) {
        best = ms;
        keep = c;
      }
    }
    plan->threads2 = keep.threads;
    plan->args2.batch_th = keep.batch_th;
    plan->args2.batch_ph = keep.batch_ph;
    plan->smem2 = keep.smem;
  }
  cudaEventDestroy(e0);
  cudaEventDestroy(e1);
  if (best_ms) *best_ms = best;
  return st;
}

}  // extern "C"
