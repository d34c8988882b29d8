// CUDA graph construction for the device-driven loops.
//
// Every iterative part of the solve (the outer flexible CG, and the batched
// inner PCG of each degree level inside the preconditioner) runs as a
// conditional WHILE node of a CUDA graph: a kernel inside the loop body sets
// the loop condition with cudaGraphSetConditional once it has reduced the
// convergence test, so no value travels to the host between iterations. A
// whole solve is captured once per option set and replayed with one
// cudaGraphLaunch.
#pragma once

#include <functional>
#include <map>
#include <string>

#include "sghsc_internal.cuh"

namespace sghsc {

// How a loop-control kernel reports the loop condition: through the graph's
// conditional handle (captured mode) and/or a device flag (eager mode).
struct LoopCtl {
  cudaGraphConditionalHandle cond;
  int has_cond;
  int* flag;
};

using Enqueue = std::function<int(cudaStream_t)>;
using EnqueueCond = std::function<int(cudaStream_t, const LoopCtl&)>;

// A device-controlled while loop at the current point of the work on `s`.
// `pre(s, lc)` enqueues the work that sets the initial condition; `body(bs,
// lc)` enqueues the loop body, whose last kernel sets the next condition.
// Captured mode (inside run_graph): a conditional WHILE node whose body is
// captured on a nested stream. Eager mode (environment SGHSC_EAGER=1, used to
// profile single kernels, which the profiler cannot do inside graphs with
// conditional nodes): the host runs the body while the device flag is set.
int capture_while(sg_problem* h, cudaStream_t s, const EnqueueCond& pre, const EnqueueCond& body);

// Build (once per key) and launch the graph of `build` on `launch`; in eager
// mode run `build` directly on `launch`.
int run_graph(sg_problem* h, const std::string& key, const Enqueue& build, cudaStream_t launch);

// Destroy every cached graph (after a workspace reallocation or at sg_destroy).
void clear_graphs(sg_problem* h);

}  // namespace sghsc
