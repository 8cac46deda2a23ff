// Batching engine: many generalized Stokes solves advanced in lockstep, one FGMRES iteration of
// every instance per step, every kernel of a step launched once for all instances.
//
// Each instance is a gs_ctx (its own hierarchy and Krylov workspace, resident on the device).
// A step records, per instance, the launches that gs_solve() would issue for one iteration
// (gs_slot.h), merges the recordings launch by launch into batched launches whose blocks walk a
// work list of (instance, block) pairs (gs_batch.cuh), and synchronises once.  The block
// preconditioner bodies of all instances form a fixed merged sequence that is captured once into
// a CUDA graph (the plan) and replayed every step; instances that do not apply the preconditioner
// in a step, or have left, are masked off by a device flag.  Instances join and leave between
// steps (continuous batching); the plan is rebuilt when an instance joins or when half of its
// members have left.
#include <algorithm>
#include <chrono>
#include <cstring>
#include <string>
#include <vector>

#include "gs.h"
#include "gs_kernels.h"
#include "gs_slot.h"

using namespace gs;

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

// device buffer with a pinned host mirror of the same size, grown on demand
struct Staged {
  char* d = nullptr;
  char* h = nullptr;
  size_t cap = 0;
  cudaError_t reserve(size_t bytes, cudaStream_t st) {
    if (bytes <= cap) return cudaSuccess;
    size_t ncap = cap ? cap : 1 << 16;
    while (ncap < bytes) ncap *= 2;
    cudaError_t e = cudaStreamSynchronize(st);
    if (e != cudaSuccess) return e;
    release();
    e = cudaMalloc(&d, ncap);
    if (e != cudaSuccess) { d = nullptr; return e; }
    e = cudaMallocHost(&h, ncap);
    if (e != cudaSuccess) { cudaFree(d); d = nullptr; h = nullptr; return e; }
    cap = ncap;
    return cudaSuccess;
  }
  void release() {
    if (d) cudaFree(d);
    if (h) cudaFreeHost(h);
    d = h = nullptr;
    cap = 0;
  }
};

struct Launch {
  BatchFn fn;
  size_t tab_off, work_off;
  int nwork;
  size_t smem;
};

// Merge recordings (one per instance) launch by launch: the t-th launches of all instances that
// run the same kernel become one batched launch.  Argument rows and work items are appended to
// `stage`; `slot_of[i]` tags the work items of recording i (-1: never masked).
void merge(const std::vector<const Recorder*>& recs, const std::vector<int>& slot_of, std::vector<unsigned char>& stage,
           std::vector<Launch>& out) {
  size_t steps = 0;
  for (const Recorder* r : recs) steps = std::max(steps, r->ops.size());
  std::vector<BatchFn> fns;
  std::vector<std::vector<int>> members;
  auto align16 = [&]() { stage.resize((stage.size() + 15) & ~size_t(15)); };
  for (size_t t = 0; t < steps; ++t) {
    fns.clear();
    members.clear();
    for (int i = 0; i < (int)recs.size(); ++i) {
      if (t >= recs[i]->ops.size()) continue;
      const BatchFn f = recs[i]->ops[t].fn;
      size_t g = 0;
      while (g < fns.size() && fns[g] != f) ++g;
      if (g == fns.size()) {
        fns.push_back(f);
        members.emplace_back();
      }
      members[g].push_back(i);
    }
    for (size_t g = 0; g < fns.size(); ++g) {
      Launch L{fns[g], 0, 0, 0, 0};
      align16();
      L.tab_off = stage.size();
      int nwork = 0;
      for (int i : members[g]) {
        const RecOp& o = recs[i]->ops[t];
        const size_t at = stage.size();
        stage.resize(at + o.arg_size);
        std::memcpy(stage.data() + at, recs[i]->bytes.data() + o.arg_off, o.arg_size);
        nwork += o.nblk;
        L.smem = std::max(L.smem, o.smem);
      }
      align16();
      L.work_off = stage.size();
      stage.resize(L.work_off + sizeof(WorkItem) * (size_t)nwork);
      WorkItem* w = reinterpret_cast<WorkItem*>(stage.data() + L.work_off);
      int row = 0;
      for (int i : members[g]) {
        const RecOp& o = recs[i]->ops[t];
        for (int b = 0; b < o.nblk; ++b) *w++ = WorkItem{row, b, o.nblk, slot_of[i]};
        row++;
      }
      L.nwork = nwork;
      out.push_back(L);
    }
  }
}

cudaError_t run(const std::vector<Launch>& ls, const char* dbase, const int* active, cudaStream_t st) {
  for (const Launch& L : ls) {
    cudaError_t e = L.fn(dbase + L.tab_off, reinterpret_cast<const WorkItem*>(dbase + L.work_off), L.nwork, active,
                         L.smem, st);
    if (e != cudaSuccess) return e;
  }
  return cudaSuccess;
}

struct Slot {
  gs_ctx* c = nullptr;
  long long uid = 0;  // unique per gs_engine_add: a context address may be reused after gs_destroy
  long long tag = 0;
  double t_added = 0.0;
};

}  // namespace

struct gs_engine {
  cudaStream_t st = nullptr;   // all work
  cudaStream_t cap = nullptr;  // plan capture
  int max_slots = 0, max_restart = 0;
  size_t gstride = 0, ystride = 0;  // doubles per slot in the gather / y areas
  std::vector<Slot> slots;
  // fixed area: [gather doubles | y doubles | active ints]
  Staged fixed;
  size_t off_y = 0, off_active = 0, fixed_bytes = 0;
  Staged step;  // per-step argument tables and work lists
  // plan: merged preconditioner bodies of its members, captured as a graph
  // per slot: uid of the solve whose body is in the plan (0: none).  Membership is keyed by uid,
  // not by context address, so a new context allocated where a destroyed one lived never runs
  // the old one's recorded launches.
  std::vector<long long> plan_uid;
  long long next_uid = 1;
  int plan_members = 0;
  Staged plan_tabs;
  cudaGraphExec_t plan_exec = nullptr;
  long long plan_kernels = 0;
  // recordings of the current step
  std::vector<Recorder> rpre, rpost;
  std::vector<unsigned char> stage;
  std::vector<Launch> lpre, lpost;
  std::vector<gs_engine_result> done;
  gs_engine_stats stats{};
};

namespace {

#define ECK(...)                                                                                  \
  do {                                                                                            \
    cudaError_t e__ = (__VA_ARGS__);                                                              \
    if (e__ != cudaSuccess) return report(GS_ECUDA, std::string(#__VA_ARGS__) + ": " + cudaGetErrorString(e__)); \
  } while (0)

double* gather_dev(gs_engine* e, int s) { return reinterpret_cast<double*>(e->fixed.d) + (size_t)s * e->gstride; }
double* gather_host(gs_engine* e, int s) { return reinterpret_cast<double*>(e->fixed.h) + (size_t)s * e->gstride; }
double* y_dev(gs_engine* e, int s) { return reinterpret_cast<double*>(e->fixed.d + e->off_y) + (size_t)s * e->ystride; }
double* y_host(gs_engine* e, int s) { return reinterpret_cast<double*>(e->fixed.h + e->off_y) + (size_t)s * e->ystride; }
int* active_dev(gs_engine* e) { return reinterpret_cast<int*>(e->fixed.d + e->off_active); }
int* active_host(gs_engine* e) { return reinterpret_cast<int*>(e->fixed.h + e->off_active); }

void drop_plan(gs_engine* e) {
  if (e->plan_exec) cudaGraphExecDestroy(e->plan_exec);
  e->plan_exec = nullptr;
  std::fill(e->plan_uid.begin(), e->plan_uid.end(), 0);
  e->plan_members = 0;
  e->plan_kernels = 0;
}

// Rebuild the plan from the preconditioner bodies of every occupied slot.
gs_status build_plan(gs_engine* e) {
  ECK(cudaStreamSynchronize(e->st));  // the old plan's tables may be in use
  drop_plan(e);
  std::vector<const Recorder*> recs;
  std::vector<int> slot_of;
  for (int s = 0; s < e->max_slots; ++s) {
    gs_ctx* c = e->slots[s].c;
    if (!c) continue;
    gs_status st;
    const Recorder* r = slot_body(c, &st);
    if (!r) return st;
    recs.push_back(r);
    slot_of.push_back(s);
    e->plan_uid[s] = e->slots[s].uid;
  }
  e->plan_members = (int)recs.size();
  if (recs.empty()) return GS_OK;
  std::vector<unsigned char> stage;
  std::vector<Launch> ls;
  merge(recs, slot_of, stage, ls);
  ECK(e->plan_tabs.reserve(stage.size(), e->st));
  std::memcpy(e->plan_tabs.h, stage.data(), stage.size());
  ECK(cudaMemcpyAsync(e->plan_tabs.d, e->plan_tabs.h, stage.size(), cudaMemcpyHostToDevice, e->st));
  ECK(cudaStreamSynchronize(e->st));
  const long long before = launches_total();
  ECK(cudaStreamBeginCapture(e->cap, cudaStreamCaptureModeRelaxed));
  cudaError_t le = run(ls, e->plan_tabs.d, active_dev(e), e->cap);
  cudaGraph_t graph = nullptr;
  cudaError_t ce = cudaStreamEndCapture(e->cap, &graph);
  e->plan_kernels = launches_total() - before;
  launched(cudaSuccess, (int)-e->plan_kernels);  // captured, not run
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    drop_plan(e);
    return report(GS_ECUDA, std::string("plan capture: ") + cudaGetErrorString(le != cudaSuccess ? le : ce));
  }
  cudaError_t ie = cudaGraphInstantiate(&e->plan_exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) {
    e->plan_exec = nullptr;
    drop_plan(e);
    return report(GS_ECUDA, std::string("plan instantiate: ") + cudaGetErrorString(ie));
  }
  e->stats.plan_builds++;
  return GS_OK;
}

gs_status engine_step(gs_engine* e, int* n_active) {
  // plan: every slot that applies the preconditioner this step must be in it with its context
  bool rebuild = false;
  int stale = 0, occupied = 0;
  for (int s = 0; s < e->max_slots; ++s) {
    gs_ctx* c = e->slots[s].c;
    const bool member = c && e->plan_uid[s] == e->slots[s].uid;
    if (c) occupied++;
    if (e->plan_uid[s] != 0 && !member) stale++;
    if (c && !member && slot_wants_body(c)) rebuild = true;
  }
  if (e->plan_members > 0 && 2 * stale > e->plan_members) rebuild = true;
  if (rebuild) {
    gs_status st = build_plan(e);
    if (st != GS_OK) return st;
  }
  // record this step's launches of every occupied slot
  std::vector<const Recorder*> pre, post;
  std::vector<int> slot_of_pre, slot_of_post;
  Recorder* prev = current_recorder();
  int any_body = 0;
  for (int s = 0; s < e->max_slots; ++s) {
    gs_ctx* c = e->slots[s].c;
    int* act = active_host(e) + s;
    *act = 0;
    if (!c) continue;
    const bool body = slot_wants_body(c);
    if (body && e->plan_uid[s] == e->slots[s].uid) *act = 1;
    any_body |= *act;
    Recorder& rp = e->rpre[s];
    Recorder& rq = e->rpost[s];
    rp.clear();
    rq.clear();
    current_recorder() = &rp;
    gs_status st = slot_record_pre(c);
    if (st == GS_OK) {
      current_recorder() = &rq;
      st = slot_record_post(c, gather_dev(e, s));
    }
    current_recorder() = prev;
    if (st != GS_OK) return st;
    pre.push_back(&rp);
    slot_of_pre.push_back(-1);
    post.push_back(&rq);
    slot_of_post.push_back(-1);
  }
  e->stage.clear();
  e->lpre.clear();
  e->lpost.clear();
  merge(pre, slot_of_pre, e->stage, e->lpre);
  merge(post, slot_of_post, e->stage, e->lpost);
  ECK(e->step.reserve(e->stage.size() + 16, e->st));
  if (!e->stage.empty()) {
    std::memcpy(e->step.h, e->stage.data(), e->stage.size());
    ECK(cudaMemcpyAsync(e->step.d, e->step.h, e->stage.size(), cudaMemcpyHostToDevice, e->st));
  }
  // y vectors staged by the previous step's host phase, and the plan's activity flags
  ECK(cudaMemcpyAsync(e->fixed.d + e->off_y, e->fixed.h + e->off_y, e->fixed_bytes - e->off_y, cudaMemcpyHostToDevice,
                      e->st));
  ECK(run(e->lpre, e->step.d, nullptr, e->st));
  if (any_body && e->plan_exec) {
    ECK(cudaGraphLaunch(e->plan_exec, e->st));
    launched(cudaSuccess, (int)e->plan_kernels);
  }
  ECK(run(e->lpost, e->step.d, nullptr, e->st));
  ECK(cudaMemcpyAsync(e->fixed.h, e->fixed.d, e->off_y, cudaMemcpyDeviceToHost, e->st));
  ECK(cudaStreamSynchronize(e->st));
  e->stats.steps++;
  e->stats.batched_launches += (long long)(e->lpre.size() + e->lpost.size());
  // host phase
  int still = 0;
  for (int s = 0; s < e->max_slots; ++s) {
    gs_ctx* c = e->slots[s].c;
    if (!c) continue;
    gs_status st = slot_update(c, gather_host(e, s), y_host(e, s), y_dev(e, s));
    if (st != GS_OK) return st;
    gs_engine_result r{};
    if (slot_done(c, &r.status, &r.iterations, &r.rel_residual)) {
      r.tag = e->slots[s].tag;
      r.t_added = e->slots[s].t_added;
      r.t_done = now_s();
      e->done.push_back(r);
      e->slots[s].c = nullptr;
      e->stats.completed++;
    } else {
      still++;
    }
  }
  if (n_active) *n_active = still;
  (void)occupied;
  return GS_OK;
}

}  // namespace

extern "C" {

gs_status gs_engine_create(int max_slots, int max_restart, void* stream, gs_engine** out) {
  if (!out) return report(GS_EINVAL, "out is NULL");
  *out = nullptr;
  if (max_slots < 1 || max_slots > 65536) return report(GS_EINVAL, "max_slots must be in [1, 65536]");
  if (max_restart <= 0) max_restart = 50;
  gs_engine* e = new gs_engine();
  e->st = (cudaStream_t)stream;
  e->max_slots = max_slots;
  e->max_restart = max_restart;
  e->gstride = (size_t)((slot_gather_max(max_restart) + 3) & ~3);
  e->ystride = (size_t)((max_restart + 3) & ~3);
  e->slots.assign(max_slots, Slot());
  e->plan_uid.assign(max_slots, 0);
  e->rpre.resize(max_slots);
  e->rpost.resize(max_slots);
  e->off_y = sizeof(double) * e->gstride * max_slots;
  e->off_active = e->off_y + sizeof(double) * e->ystride * max_slots;
  e->fixed_bytes = e->off_active + sizeof(int) * (size_t)max_slots;
  cudaError_t ce = cudaStreamCreateWithFlags(&e->cap, cudaStreamNonBlocking);
  if (ce == cudaSuccess) ce = e->fixed.reserve(e->fixed_bytes, e->st);
  if (ce != cudaSuccess) {
    if (e->cap) cudaStreamDestroy(e->cap);
    e->fixed.release();
    delete e;
    return report(GS_ECUDA, std::string("engine buffers: ") + cudaGetErrorString(ce));
  }
  std::memset(e->fixed.h, 0, e->fixed.cap);
  *out = e;
  return GS_OK;
}

gs_status gs_engine_add(gs_engine* e, gs_ctx* c, const double* rhs, double* x, double tol, long long tag) {
  if (!e || !c) return report(GS_EINVAL, "NULL engine or context");
  if (slot_restart(c) > e->max_restart) return report(GS_EINVAL, "context restart exceeds the engine's max_restart");
  int free_slot = -1;
  for (int s = 0; s < e->max_slots; ++s) {
    if (e->slots[s].c == c) return report(GS_EINVAL, "context is already in the engine");
    if (!e->slots[s].c && free_slot < 0) free_slot = s;
  }
  if (free_slot < 0) return report(GS_EBUSY, "no free slot");
  gs_status st = slot_begin(c, rhs, x, tol);
  if (st != GS_OK) return st;
  // the engine's stream does not wait on the context's stream: finish what is queued there
  ECK(cudaStreamSynchronize(slot_stream(c)));
  e->slots[free_slot].c = c;
  e->slots[free_slot].uid = e->next_uid++;
  e->slots[free_slot].tag = tag;
  e->slots[free_slot].t_added = now_s();
  return GS_OK;
}

gs_status gs_engine_step(gs_engine* e, int* active) {
  if (!e) return report(GS_EINVAL, "engine is NULL");
  return engine_step(e, active);
}

int gs_engine_poll(gs_engine* e, gs_engine_result* out, int max) {
  if (!e || max <= 0 || !out) return 0;
  const int n = std::min((int)e->done.size(), max);
  for (int i = 0; i < n; ++i) out[i] = e->done[i];
  e->done.erase(e->done.begin(), e->done.begin() + n);
  return n;
}

int gs_engine_active(const gs_engine* e) {
  if (!e) return 0;
  int n = 0;
  for (const Slot& s : e->slots) n += s.c ? 1 : 0;
  return n;
}

gs_status gs_engine_get_stats(const gs_engine* e, gs_engine_stats* out) {
  if (!e || !out) return report(GS_EINVAL, "NULL argument");
  *out = e->stats;
  out->plan_kernels = e->plan_kernels;
  return GS_OK;
}

void gs_engine_destroy(gs_engine* e) {
  if (!e) return;
  cudaStreamSynchronize(e->st);
  drop_plan(e);
  e->plan_tabs.release();
  e->step.release();
  e->fixed.release();
  if (e->cap) cudaStreamDestroy(e->cap);
  delete e;
}

}  // extern "C"
