// trace.cu -- the task trace of the streamed pipelines and the NVTX ranges of
// the host-side stages.
//
// Sec. IV-C keeps copies, GPU work and host work in flight at once on
// dedicated threads and offers an optional profiling flag that records the
// tasks each of them executes (Fig. 4 shows such a trace on a timeline).
// Here the resources are CUDA streams: with tracing on, every task of the
// out-of-core and load-and-run pipelines is bracketed by two CUDA events on
// the stream that runs it, so the timeline comes from the device clock
// without synchronising the pipeline.
#include <cuda_runtime.h>
#include <nvtx3/nvToolsExt.h>

#include "ap_internal.h"

namespace ap {

void Tracer::clear() {
  for (TraceRec &r : recs) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
  }
  recs.clear();
  if (base) cudaEventDestroy(base);
  base = nullptr;
}

cudaError_t Tracer::start(cudaStream_t s) {
  if (!on) return cudaSuccess;
  clear();
  cudaError_t e = cudaEventCreate(&base);
  if (e == cudaSuccess) e = cudaEventRecord(base, s);
  return e;
}

int Tracer::begin(int32_t stream, int32_t stage, int64_t index, uint64_t bytes,
                  cudaStream_t st) {
  if (!on || !base) return -1;
  TraceRec r;
  r.stream = stream;
  r.stage = stage;
  r.index = index;
  r.bytes = bytes;
  if (cudaEventCreate(&r.a) != cudaSuccess || cudaEventCreate(&r.b) != cudaSuccess ||
      cudaEventRecord(r.a, st) != cudaSuccess) {
    if (r.a) cudaEventDestroy(r.a);
    if (r.b) cudaEventDestroy(r.b);
    cudaGetLastError();
    return -1;
  }
  recs.push_back(r);
  return (int)recs.size() - 1;
}

void Tracer::end(int rec, cudaStream_t st) {
  if (rec < 0 || rec >= (int)recs.size()) return;
  if (cudaEventRecord(recs[rec].b, st) != cudaSuccess) cudaGetLastError();
}

NvtxRange::NvtxRange(const char *name) { nvtxRangePushA(name); }
NvtxRange::~NvtxRange() { nvtxRangePop(); }

}  // namespace ap

using namespace ap;

extern "C" ap_status ap_set_trace(ap_items *it, int32_t on) {
  if (!it || (on != 0 && on != 1)) return AP_ERR_INVALID_ARG;
  it->trace.on = on != 0;
  if (!it->trace.on) it->trace.clear();
  return AP_OK;
}

extern "C" ap_status ap_get_trace(ap_items *it, ap_trace_event *out, int64_t cap,
                                  int64_t *count) {
  if (!it || !count || (cap > 0 && !out)) return AP_ERR_INVALID_ARG;
  Tracer &tr = it->trace;
  *count = (int64_t)tr.recs.size();
  for (int64_t k = 0; k < *count && k < cap; ++k) {
    const TraceRec &r = tr.recs[k];
    float a = 0.f, b = 0.f;
    AP_TRY(cudaEventSynchronize(r.b));
    AP_TRY(cudaEventElapsedTime(&a, tr.base, r.a));
    AP_TRY(cudaEventElapsedTime(&b, tr.base, r.b));
    out[k].stream = r.stream;
    out[k].stage = r.stage;
    out[k].index = r.index;
    out[k].bytes = r.bytes;
    out[k].start_ms = a;
    out[k].end_ms = b;
  }
  return AP_OK;
}
