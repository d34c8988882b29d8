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

using Enqueue = std::function<int(cudaStream_t)>;
using EnqueueCond = std::function<int(cudaStream_t, cudaGraphConditionalHandle)>;

// Inside an active capture on `s`: create a WHILE node at the current point.
// `pre(s, cond)` enqueues (on s, before the node) the work that sets the
// initial condition; `body(bs, cond)` enqueues the loop body on a nested
// capture stream. Capture then continues on `s` after the node.
int capture_while(sg_problem* h, cudaStream_t s, const EnqueueCond& pre, const EnqueueCond& body);

// Build (once per key) and launch the graph of `build` on `launch`.
int run_graph(sg_problem* h, const std::string& key, const Enqueue& build, cudaStream_t launch);

// Destroy every cached graph (after a workspace reallocation or at sg_destroy).
void clear_graphs(sg_problem* h);

}  // namespace sghsc
