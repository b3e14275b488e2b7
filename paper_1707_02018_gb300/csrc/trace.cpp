// Optional per-kernel timing.  When armed, every kernel this library launches
// is bracketed by a pair of CUDA events recorded on the launch stream, so a
// caller can read each kernel's device time afterwards without a profiler.
// Disarmed (the default) it costs one branch per launch.  Tracing is meant
// for one host thread at a time.
#include <vector>

#include "adjwt_internal.h"

namespace adjwt {
namespace {

struct Rec {
  const char* name;
  int tag;
  cudaEvent_t a, b;
};

std::vector<Rec> g_pool;
int g_used = 0;
bool g_on = false;

}  // namespace

int trace_begin(const char* name, int tag, cudaStream_t s) {
  if (!g_on || g_used >= static_cast<int>(g_pool.size())) return -1;
  Rec& r = g_pool[g_used];
  r.name = name;
  r.tag = tag;
  if (cudaEventRecord(r.a, s) != cudaSuccess) return -1;
  return g_used++;
}

void trace_end(int id, cudaStream_t s) {
  if (id >= 0) cudaEventRecord(g_pool[id].b, s);
}

}  // namespace adjwt

using namespace adjwt;

extern "C" int adjwt_trace_enable(int capacity) {
  for (Rec& r : g_pool) {
    cudaEventDestroy(r.a);
    cudaEventDestroy(r.b);
  }
  g_pool.clear();
  g_used = 0;
  g_on = false;
  if (capacity <= 0) return ADJWT_OK;
  g_pool.resize(capacity);
  for (Rec& r : g_pool) {
    r.name = "";
    r.tag = 0;
    ADJWT_CUDA_CHECK(cudaEventCreate(&r.a));
    ADJWT_CUDA_CHECK(cudaEventCreate(&r.b));
  }
  g_on = true;
  return ADJWT_OK;
}

extern "C" int adjwt_trace_count(void) { return g_used; }

extern "C" int adjwt_trace_reset(void) {
  g_used = 0;
  return ADJWT_OK;
}

extern "C" int adjwt_trace_get(int i, const char** name, int* tag, float* ms) {
  if (i < 0 || i >= g_used) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_trace_get: index out of range");
  Rec& r = g_pool[i];
  ADJWT_CUDA_CHECK(cudaEventSynchronize(r.b));
  float t = 0.0f;
  ADJWT_CUDA_CHECK(cudaEventElapsedTime(&t, r.a, r.b));
  if (name) *name = r.name;
  if (tag) *tag = r.tag;
  if (ms) *ms = t;
  return ADJWT_OK;
}

// Device time from the start of record `first` to the end of record `last`
// (both on one stream, first <= last): a whole multi-kernel operator call,
// launch gaps included.
extern "C" int adjwt_trace_span(int first, int last, float* ms) {
  if (first < 0 || last < first || last >= g_used || !ms)
    return fail(ADJWT_ERR_INVALID_ARG, "adjwt_trace_span: indices out of range or ms NULL");
  ADJWT_CUDA_CHECK(cudaEventSynchronize(g_pool[last].b));
  ADJWT_CUDA_CHECK(cudaEventElapsedTime(ms, g_pool[first].a, g_pool[last].b));
  return ADJWT_OK;
}
