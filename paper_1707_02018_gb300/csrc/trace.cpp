// Optional device timing without a profiler.  When armed at level 1 (the
// default) every kernel this library launches is bracketed by a pair of CUDA
// events recorded on the launch stream; at level 2 only whole operator calls
// of the FISTA step and the channel gradient are (W, R^*(R u - b), W^* with
// the prox, the momentum update, the channel gradient), so that the events
// leave the launches inside an operator back to back (programmatic dependent
// launch overlaps them as in an untraced call).  Disarmed it costs one branch
// per launch.  Tracing is meant for one host thread at a time.
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
int g_level = 1;  // 1: every kernel; 2: whole operator calls

int record(int level, const char* name, int tag, cudaStream_t s) {
  if (!g_on || g_level != level || g_used >= static_cast<int>(g_pool.size())) return -1;
  Rec& r = g_pool[g_used];
  r.name = name;
  r.tag = tag;
  if (cudaEventRecord(r.a, s) != cudaSuccess) return -1;
  return g_used++;
}

}  // namespace

int trace_begin(const char* name, int tag, cudaStream_t s) { return record(1, name, tag, s); }
int trace_op_begin(const char* name, int tag, cudaStream_t s) { return record(2, name, tag, s); }

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

extern "C" int adjwt_trace_set_level(int level) {
  if (level != 1 && level != 2) return fail(ADJWT_ERR_INVALID_ARG, "adjwt_trace_set_level: level must be 1 or 2");
  g_level = level;
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
