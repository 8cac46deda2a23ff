// Resumable FGMRES of one context, driven by the batching engine (internal to libgs.so).
//
// The solve of gs_solve() split at its host synchronisation points.  Every engine step, for each
// instance: slot_record_pre() records the launches that precede the preconditioner body, the
// engine runs the merged preconditioner bodies, slot_record_post() records the launches that
// follow it (ending with a gather of the scalars the host needs), the engine synchronises once,
// and slot_update() applies the Givens rotations and picks the next phase.  The recorded launches
// are the ones gs_solve() issues (same kernels, same arguments, same order), with classical
// Gram-Schmidt applied twice.
#pragma once
#include <string>

#include "gs.h"
#include "gs_kernels.h"

namespace gs {

// set the thread's last-error text (gs_last_error) and return s
gs_status report(gs_status s, const std::string& why);

// number of doubles slot_record_post() gathers at most (restart m)
inline int slot_gather_max(int m) { return 2 * (m + 2) + 4; }

// Validate the context for engine use and reset its solve state.  b, x: device, full length;
// x holds the initial guess.
gs_status slot_begin(gs_ctx* c, const double* b, double* x, double tol);
// Record the preconditioner body once (cached in the context); later calls return the cache.
const Recorder* slot_body(gs_ctx* c, gs_status* st);
// true when the next step applies the preconditioner (the body must run for this slot)
bool slot_wants_body(const gs_ctx* c);
// Record this step's launches before / after the preconditioner body (a Recorder must be
// installed on the calling thread).  gather_dev: device area of slot_gather_max() doubles.
gs_status slot_record_pre(gs_ctx* c);
gs_status slot_record_post(gs_ctx* c, double* gather_dev);
// Host part of the step: gathered = host copy of the gather area.  y_host / y_dev: a host
// staging area of restart doubles and its device mirror, copied host -> device by the engine
// before the next step's launches.
gs_status slot_update(gs_ctx* c, const double* gathered, double* y_host, const double* y_dev);
// true once the solve has finished; then status, iterations and the explicit relative residual
bool slot_done(const gs_ctx* c, gs_status* status, int* iterations, double* rel_residual);
const char* slot_error(const gs_ctx* c);
int slot_restart(const gs_ctx* c);
cudaStream_t slot_stream(const gs_ctx* c);

}  // namespace gs
