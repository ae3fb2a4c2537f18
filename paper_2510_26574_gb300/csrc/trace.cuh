// Per-stage launch timing with CUDA events on the launching stream.
#pragma once
#include <cuda_runtime.h>

namespace kevd {

// Stage ids (also in include/kevd.h as KEVD_STAGE_*).
enum Stage {
    kStPropose = 0, kStGather, kStBlockH, kStReject, kStEngine, kStDegree, kStGram, kStSolver, kStLift,
    kStOther, kStProducts, kNumStages
};

// Records an event pair around the launches between begin() and end() when
// tracing is on; a no-op otherwise.  flush() (after the stream is
// synchronised) folds the elapsed times into the per-stage totals.
int trace_begin(int stage, cudaStream_t s);
void trace_end(int handle, cudaStream_t s);
void trace_flush();

struct TraceScope {
    int h;
    cudaStream_t s;
    TraceScope(int stage, cudaStream_t st) : h(trace_begin(stage, st)), s(st) {}
    ~TraceScope() { trace_end(h, s); }
};

}  // namespace kevd
