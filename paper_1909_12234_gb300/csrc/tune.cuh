// Launch-shape autotuner.
//
// A kernel with several valid launch shapes (rows per thread, right-hand
// sides per block, one or two right-hand sides per thread) asks the tuner
// which to use for a given problem key.  On the first request for a key the
// tuner times every candidate on the caller's stream (one untimed launch,
// then the best of `reps` timed launches with CUDA events) and keeps the
// fastest; later requests return the stored choice.  Candidates must be
// out-of-place kernels whose inputs the timing launches do not change.  No
// timing runs while the stream is being captured into a graph or when
// tuning is off: then the first applicable candidate (the default) is used.
#pragma once

#include <functional>
#include <string>

#include "qd_internal.cuh"

namespace qd {

// launch(c) enqueues candidate c on ctx.stream and returns false (having
// enqueued nothing) when c does not apply to this problem.  Returns the
// chosen candidate, whose launch the caller then makes itself.
int tune_pick(qd_ctx& ctx, const std::string& key, int ncand, const std::function<bool(int)>& launch);

// The stored (or forced) choice for key without timing anything; -1: none.
int tune_lookup(const std::string& key);
// Whether tune_pick would time candidates now (tuning on, no forced
// candidate, the stream not being captured).
bool tune_can_time(qd_ctx& ctx);

// 0: defaults only; 1: tune on first use (the library's default).
void tune_set_mode(int mode);
// >= 0: tune_pick returns this candidate (when < ncand) without timing;
// -1: normal selection.
void tune_force(int candidate);
int tune_mode();
// The table as text, one line per key: key, chosen candidate, then the
// measured time (ms) of every candidate (-1: not applicable).
std::string tune_report();
void tune_clear();

}  // namespace qd
