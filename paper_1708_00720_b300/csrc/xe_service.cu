// Streaming X-engine service: several independent streams of gulps, each with
// a device ring, correlated and integrated as the gulps arrive.
//
// The paper's runtime model ("Memory management and ring buffers",
// "Guarantees"): a writer fills a ring in gulps; the ring holds a buffer
// factor of gulps; a guaranteed reader makes the writer wait when the ring is
// full (back-pressure), an unguaranteed one lets data be skipped.  Here the
// writer is the host capture side (xe_service_reserve / xe_service_commit),
// the reader is the X-engine, and integration spans a fixed number of gulps
// (the paper's accumulate block).
//
// Per stream:
//   pinned host staging ring  [R][T][C][N]  (the writer fills a slot)
//   device ring               [R][T][C][N]  (H2D copy of each committed slot)
//   plan (int32 accumulator), device visibility buffer, two pinned output slots
//   three CUDA streams: H2D copies, compute (correlate, integrate), D2H copies
// Host-link copies (a committed gulp into its device slot, an integration's
// visibilities out) go in 32 MB pieces, at most 4 in flight per direction,
// the streams' queued copies taking turns, so that a small stream's copy does
// not wait behind a large one's (copies of one direction run in submission
// order); a gulp is dispatched once its last piece has been issued.  The dispatcher
// launches the correlation of every pending gulp that is contiguous in the
// ring and belongs to the current integration as ONE launch, as soon as the
// stream has fewer than two launches in flight and the GPU fewer than two in
// all: with an idle GPU each gulp goes alone (lowest latency); with a busy
// GPU gulps queue up and go together (fewer, larger launches), and the runs
// of several e4m3 streams that are ready at once share one launch of the
// pair kernel (xe_correlate_batch).  When an integration's last gulp has been dispatched (or
// on flush) the accumulator is emitted into a free output slot and copied to
// host memory; completion times come from host callbacks enqueued after the
// copies.  Ring slots are recycled when the launch that read them completes.
//
// Host-side fault injection: XE_FAULT_LAUNCH makes the stream's next launch
// fail as a failing CUDA call would (the stream enters the failed state, other
// streams continue); XE_FAULT_DROP_GULP loses the next committed gulp in
// transit (its integration reports it as skipped).
//
// A dry-run mode (XE_SERVICE_DRYRUN) runs the same bookkeeping with no CUDA
// calls, so the host logic is testable without a GPU; with XE_SERVICE_MANUAL
// the dry-run work stays "in flight" until xe_service_dryrun_complete.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstdint>
#include <cstdlib>
#include <cstring>
#include <deque>
#include <memory>
#include <mutex>
#include <new>
#include <string>
#include <thread>
#include <vector>

#include "xengine.h"
#include "xe_kernels.h"

namespace {

using Clock = std::chrono::steady_clock;

double now_ms() {
  return std::chrono::duration<double, std::milli>(Clock::now().time_since_epoch()).count();
}

constexpr int kOutSlots = 2;     // pinned output buffers per stream
constexpr int kMaxInflight = 2;  // correlate launches in flight per stream
// ... and on the whole GPU: with the GPU busy, further ready gulps wait and
// then go together, several streams in one launch (with it idle, a gulp
// goes at once, alone)
#ifndef XE_SVC_INFLIGHT_TOTAL
#define XE_SVC_INFLIGHT_TOTAL 2
#endif
constexpr int kMaxInflightTotal = XE_SVC_INFLIGHT_TOTAL;
// Host-link copies go out in pieces, a bounded number in flight per
// direction and the streams taking turns: a GPU runs the copies of one
// direction in submission order, so a 1 GB visibility copy issued whole
// would hold a small stream's copy back for ~20 ms.  A piece's completion
// is an event the worker polls (a host callback per piece would hold its
// CUDA stream until it had run, leaving gaps between pieces).
#ifndef XE_SVC_COPY_PIECE_MB
#define XE_SVC_COPY_PIECE_MB 32
#endif
#ifndef XE_SVC_COPY_PIECES
#define XE_SVC_COPY_PIECES 4
#endif
constexpr size_t kCopyPiece = size_t(XE_SVC_COPY_PIECE_MB) << 20;
constexpr int kPiecesInFlight = XE_SVC_COPY_PIECES;

enum SlotState : int { kFree = 0, kReserved, kCommitted, kDispatched };

struct Gulp {
  long long seq;
  int slot;
  double t_commit;
  cudaEvent_t h2d_done;   // recorded after the slot's last H2D piece (real mode)
  bool h2d_issued;        // every piece of its H2D copy has been issued
};

struct Batch {
  int first_slot = 0, n = 0;
  cudaEvent_t done = nullptr;
  std::atomic<int> complete{0};
  bool counts = false;   // the one batch of its launch that holds the service's in-flight count
};

// Gulps of one stream ready to go in one launch (see next_run).
struct Run {
  int first = 0, n = 0;   // ring slots [first, first + n)
  long long integ = 0;    // integration they belong to
  bool accumulate = false;
};

struct Emit {
  long long index = 0, first_seq = 0;
  int gulps = 0, skipped = 0;
  long long samples = 0;
  double t_last_commit = 0;
  int out_slot = -1;
  int status = XE_OK;
  std::atomic<int> ready{0};
  double t_done = 0;
};

struct ServiceImpl;

// One host-link copy, issued piece by piece by pump_copies: a gulp into its
// ring slot (H2D) or an integration's visibilities out (D2H).
struct CopyJob {
  uint8_t* dst = nullptr;
  const uint8_t* src = nullptr;
  size_t bytes = 0, issued = 0;
  long long gulp_seq = -1;   // H2D: the gulp it carries
  Emit* emit = nullptr;      // D2H: the integration it delivers
};

struct StreamImpl {
  int id = 0;
  xe_stream_config cfg{};
  ServiceImpl* svc = nullptr;
  size_t gulp_bytes = 0, vis_bytes = 0;
  long long dev_bytes = 0, host_bytes = 0;
  // resources
  xe_plan_t plan = nullptr;
  uint8_t* h_ring = nullptr;
  uint8_t* d_ring = nullptr;
  void* d_vis = nullptr;
  void* h_out[kOutSlots] = {nullptr, nullptr};
  bool out_busy[kOutSlots] = {false, false};
  cudaStream_t s_h2d = nullptr, s_comp = nullptr, s_d2h = nullptr;
  cudaEvent_t d2h_done = nullptr;   // last D2H out of d_vis
  std::deque<std::unique_ptr<CopyJob>> copies[2];   // H2D, D2H jobs of this stream, in order
  bool d2h_open = false;            // a D2H job out of d_vis still has pieces to issue
  // ring state
  std::vector<int> slot_state;
  std::vector<cudaEvent_t> slot_event;
  int next_slot = 0;                 // where the writer reserves next (ring order)
  int reserved_slot = -1;
  std::deque<Gulp> pending;          // committed, not yet dispatched (commit order)
  std::deque<std::unique_ptr<Batch>> inflight;
  // integration state
  long long integ_index = -1;        // integration the accumulator belongs to (-1: none)
  int integ_gulps = 0;
  long long integ_samples = 0;
  double integ_t_last = 0;
  bool integ_has_data = false;       // a launch with accumulate = 0 has been made for it
  bool emit_pending = false;         // integration complete, waiting to be emitted
  long long emit_index = 0;
  long long flush_seq = -1;          // gulps up to this one have been flushed
  long long last_seq = -1;
  std::deque<std::unique_ptr<Emit>> emits;   // emitted, in order (ready or not)
  std::deque<std::unique_ptr<Emit>> handed;  // returned by poll, output slot not yet released
  // faults
  int fault = 0;
  int state = XE_OK;
  // cross-stream launches
  cudaEvent_t comp_mark = nullptr;   // recorded on s_comp before a shared launch
  // stats
  xe_stream_stats st{};
};

struct ServiceImpl {
  long long cap = 0, used = 0;
  int flags = 0;
  bool batch = true;     // ready gulps of several e4m3 streams share one launch
  int inflight_total = 0;   // launches in flight on the GPU (a shared launch counts once)
  cudaStream_t s_batch = nullptr;   // the shared launches
  int num_sms = 148;   // of the service's device; a dry run models a 148-SM B300
  bool dry = false, manual = false;
  std::mutex mu;
  std::condition_variable cv;
  std::vector<std::unique_ptr<StreamImpl>> streams;
  std::thread worker;
  bool stop = false;
  std::string last_error;
  // per direction (H2D, D2H): the events of the pieces in flight, oldest
  // first, and the stream whose job goes next
  std::deque<cudaEvent_t> pieces[2];
  int copy_turn[2] = {0, 0};
};

struct HostCbBatch {
  Batch* b;
  ServiceImpl* svc;
};
struct HostCbEmit {
  Emit* e;
  ServiceImpl* svc;
};
struct HostCbShared {
  std::vector<Batch*> b;
  ServiceImpl* svc;
};


void CUDART_CB on_batch_done(void* p) {
  auto* h = static_cast<HostCbBatch*>(p);
  h->b->complete.store(1, std::memory_order_release);
  h->svc->cv.notify_all();
  delete h;
}

void CUDART_CB on_shared_done(void* p) {
  auto* h = static_cast<HostCbShared*>(p);
  for (Batch* b : h->b) b->complete.store(1, std::memory_order_release);
  h->svc->cv.notify_all();
  delete h;
}

void CUDART_CB on_emit_done(void* p) {
  auto* h = static_cast<HostCbEmit*>(p);
  h->e->t_done = now_ms();
  h->e->ready.store(1, std::memory_order_release);
  h->svc->cv.notify_all();
  delete h;
}

xe_status fail_stream(StreamImpl* s, xe_status st, const char* what) {
  s->state = st;
  s->svc->last_error = std::string("stream ") + std::to_string(s->id) + ": " + what;
  return st;
}

// Retire finished launches (free their ring slots).
void retire(StreamImpl* s) {
  while (!s->inflight.empty() && s->inflight.front()->complete.load(std::memory_order_acquire)) {
    Batch* b = s->inflight.front().get();
    for (int k = 0; k < b->n; ++k) s->slot_state[(b->first_slot + k) % s->cfg.ring_gulps] = kFree;
    if (b->counts) s->svc->inflight_total--;
    if (b->done) cudaEventDestroy(b->done);
    s->inflight.pop_front();
  }
}

// Issue copy pieces while fewer than kPiecesInFlight of a direction are in
// flight, the streams with queued jobs taking turns (a stream's own jobs go
// in order, on its own CUDA stream).  A job's last piece records what waits
// for it: for a gulp, the event its correlation waits on (the gulp becomes
// dispatchable); for an integration, d2h_done and the callback that hands it
// to the consumer.
void pump_copies(ServiceImpl* svc) {
  const int ns = static_cast<int>(svc->streams.size());
  if (svc->dry || ns == 0) return;
  for (int dir = 0; dir < 2; ++dir) {
    // retire the pieces that have landed (in order: one engine per direction)
    while (!svc->pieces[dir].empty()) {
      const cudaError_t q = cudaEventQuery(svc->pieces[dir].front());
      if (q == cudaErrorNotReady) break;
      if (q != cudaSuccess) cudaGetLastError();
      cudaEventDestroy(svc->pieces[dir].front());
      svc->pieces[dir].pop_front();
    }
    int idle = 0;
    while (idle < ns && static_cast<int>(svc->pieces[dir].size()) < kPiecesInFlight) {
      const int turn = svc->copy_turn[dir] % ns;
      svc->copy_turn[dir] = (turn + 1) % ns;
      StreamImpl* s = svc->streams[turn].get();
      if (s->copies[dir].empty()) {
        ++idle;
        continue;
      }
      idle = 0;
      CopyJob* j = s->copies[dir].front().get();
      cudaStream_t cs = dir == 0 ? s->s_h2d : s->s_d2h;
      // with one stream there is nobody to take turns with: the whole copy
      const size_t n = ns == 1 ? j->bytes - j->issued : std::min(kCopyPiece, j->bytes - j->issued);
      bool ok = cudaMemcpyAsync(j->dst + j->issued, j->src + j->issued, n,
                                dir == 0 ? cudaMemcpyHostToDevice : cudaMemcpyDeviceToHost, cs) == cudaSuccess;
      if (ok) {
        cudaEvent_t pe = nullptr;
        ok = cudaEventCreateWithFlags(&pe, cudaEventDisableTiming) == cudaSuccess &&
             cudaEventRecord(pe, cs) == cudaSuccess;
        if (ok) {
          svc->pieces[dir].push_back(pe);
        } else if (pe) {
          cudaEventDestroy(pe);
        }
      }
      j->issued += n;
      if (ok && j->issued < j->bytes) continue;
      // the job's last piece has been issued (or a piece failed)
      if (dir == 0) {
        for (Gulp& g : s->pending) {
          if (g.seq != j->gulp_seq) continue;
          if (ok) ok = cudaEventRecord(g.h2d_done, cs) == cudaSuccess;
          g.h2d_issued = true;
          break;
        }
        if (!ok) {
          cudaGetLastError();
          fail_stream(s, XE_ERR_CUDA, "H2D copy failed");
        }
      } else {
        Emit* e = j->emit;
        if (ok) ok = cudaEventRecord(s->d2h_done, cs) == cudaSuccess;
        if (ok) {
          auto* cb = new HostCbEmit{e, svc};
          if (cudaLaunchHostFunc(cs, on_emit_done, cb) != cudaSuccess) {
            delete cb;
            ok = false;
          }
        }
        if (!ok) {
          cudaGetLastError();
          e->status = XE_ERR_CUDA;
          e->t_done = now_ms();
          e->ready.store(1, std::memory_order_release);
          fail_stream(s, XE_ERR_CUDA, "D2H copy failed");
        }
        s->d2h_open = false;
      }
      s->copies[dir].pop_front();
    }
  }
}

int free_out_slot(StreamImpl* s) {
  for (int k = 0; k < kOutSlots; ++k)
    if (!s->out_busy[k]) return k;
  return -1;
}

// Emit the accumulator of the current integration into a free output slot.
// Returns false if no output slot is free (the emit stays pending).
bool try_emit(StreamImpl* s) {
  if (s->d2h_open) return false;   // the previous copy out of d_vis still has pieces to issue
  const int slot = free_out_slot(s);
  if (slot < 0) return false;
  auto e = std::make_unique<Emit>();
  e->index = s->emit_index;
  e->first_seq = s->emit_index * s->cfg.integrate_gulps;
  e->gulps = s->integ_gulps;
  e->skipped = s->cfg.integrate_gulps - s->integ_gulps;
  e->samples = s->integ_samples;
  e->t_last_commit = s->integ_t_last;
  e->out_slot = slot;
  s->out_busy[slot] = true;
  Emit* raw = e.get();
  s->emits.push_back(std::move(e));
  if (s->svc->dry) {
    std::memset(s->h_out[slot], 0, s->vis_bytes);
    if (!s->svc->manual) {
      raw->t_done = now_ms();
      raw->ready.store(1);
    }
  } else {
    xe_status st = XE_OK;
    if (s->integ_has_data) {
      // d_vis is reused: wait for its previous copy-out first
      cudaStreamWaitEvent(s->s_comp, s->d2h_done, 0);
      st = xe_integrate(s->plan, s->d_vis, s->s_comp);
    } else {
      cudaMemsetAsync(s->d_vis, 0, s->vis_bytes, s->s_comp);   // an integration with no gulps at all
    }
    cudaEvent_t ev;
    cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
    cudaEventRecord(ev, s->s_comp);
    cudaStreamWaitEvent(s->s_d2h, ev, 0);   // the pieces, issued later on s_d2h, follow it
    cudaEventDestroy(ev);
    auto j = std::make_unique<CopyJob>();
    j->dst = static_cast<uint8_t*>(s->h_out[slot]);
    j->src = static_cast<const uint8_t*>(s->d_vis);
    j->bytes = s->vis_bytes;
    j->emit = raw;
    s->copies[1].push_back(std::move(j));
    s->d2h_open = true;
    if (st != XE_OK) {
      raw->status = st;
      fail_stream(s, st, "emit failed");
    }
  }
  s->st.integrations++;
  s->emit_pending = false;
  s->integ_index = -1;
  s->integ_gulps = 0;
  s->integ_samples = 0;
  s->integ_has_data = false;
  return true;
}

// The longest run of pending gulps that are contiguous in the ring and
// belong to the current integration, if the stream may launch now.
bool next_run(StreamImpl* s, Run* r) {
  if (s->state != XE_OK || s->pending.empty() || static_cast<int>(s->inflight.size()) >= kMaxInflight ||
      s->emit_pending || s->svc->inflight_total >= kMaxInflightTotal)
    return false;
  if (!s->pending.front().h2d_issued) return false;   // its copy is still being issued
  const int G = s->cfg.integrate_gulps;
  const long long integ = s->pending.front().seq / G;
  if (s->integ_index >= 0 && integ != s->integ_index) return false;   // previous integration not emitted yet
  int n = 1;
  while (n < static_cast<int>(s->pending.size()) && s->pending[n].seq / G == integ &&
         s->pending[n].slot == s->pending[n - 1].slot + 1 &&   // contiguous, no wrap
         s->pending[n].h2d_issued)
    ++n;
  r->first = s->pending.front().slot;
  r->n = n;
  r->integ = integ;
  r->accumulate = s->integ_has_data;
  return true;
}

// Bookkeeping of a run that has been launched (alone or shared).
void commit_run(StreamImpl* s, const Run& r, std::unique_ptr<Batch> b, bool shared) {
  for (int k = 0; k < r.n; ++k) {
    const Gulp& gp = s->pending.front();
    s->slot_state[gp.slot] = kDispatched;
    s->integ_t_last = gp.t_commit;
    if (gp.h2d_done) cudaEventDestroy(gp.h2d_done);
    s->pending.pop_front();
  }
  s->integ_index = r.integ;
  s->integ_gulps += r.n;
  s->integ_samples += static_cast<long long>(r.n) * s->cfg.gulp_ntime;
  s->integ_has_data = true;
  s->st.launches++;
  if (shared) s->st.shared_launches++;
  s->st.gulps_correlated += r.n;
  if (r.n > s->st.max_batch) s->st.max_batch = r.n;
  if (b->counts) s->svc->inflight_total++;
  s->inflight.push_back(std::move(b));
}

// Launch the correlation of the stream's next run on its own.
void dispatch(StreamImpl* s) {
  Run r;
  if (!next_run(s, &r)) return;
  auto b = std::make_unique<Batch>();
  b->first_slot = r.first;
  b->n = r.n;
  b->counts = true;
  if (s->fault == XE_FAULT_LAUNCH) {
    s->fault = 0;
    fail_stream(s, XE_ERR_CUDA, "injected launch failure");
    return;
  }
  if (s->svc->dry) {
    if (!s->svc->manual) b->complete.store(1);
  } else {
    cudaStreamWaitEvent(s->s_comp, s->pending[r.n - 1].h2d_done, 0);   // H2D copies are in order
    const xe_status st = xe_correlate(s->plan, s->d_ring + static_cast<size_t>(r.first) * s->gulp_bytes,
                                      r.n * s->cfg.gulp_ntime, r.accumulate ? 1 : 0, s->s_comp);
    if (st != XE_OK) {
      fail_stream(s, st, xe_plan_last_error(s->plan));
      return;
    }
    cudaEventCreateWithFlags(&b->done, cudaEventDisableTiming);
    cudaEventRecord(b->done, s->s_comp);
    if (cudaLaunchHostFunc(s->s_comp, on_batch_done, new HostCbBatch{b.get(), s->svc}) != cudaSuccess) {
      fail_stream(s, XE_ERR_CUDA, "cudaLaunchHostFunc failed");
      return;
    }
  }
  commit_run(s, r, std::move(b), false);
}

// Cross-stream batching: when two or more e4m3 streams have runs ready at the
// same time (each within one launch, at most kMaxBatch streams), they go in
// ONE launch (xe_correlate_batch) on the service's own CUDA stream, ordered
// after each stream's earlier compute work and its H2D copies; each stream's
// later work (integrate, emit) waits for the shared launch.  Streams with an
// injected fault, other operands or longer runs take the single path.
void dispatch_shared(ServiceImpl* svc) {
  StreamImpl* who[xe::kMaxBatch];
  Run runs[xe::kMaxBatch];
  int m = 0;
  for (auto& sp : svc->streams) {
    StreamImpl* s = sp.get();
    if (m == xe::kMaxBatch) break;
    retire(s);
    if (s->cfg.operand != XE_OPERAND_FP8_E4M3 || s->fault != 0) continue;
    Run r;
    if (!next_run(s, &r)) continue;
    if (static_cast<long long>(r.n) * s->cfg.gulp_ntime > 32768) continue;   // one launch per problem
    who[m] = s;
    runs[m] = r;
    ++m;
  }
  if (m < 2) return;
  std::unique_ptr<Batch> bs[xe::kMaxBatch];
  for (int k = 0; k < m; ++k) {
    bs[k] = std::make_unique<Batch>();
    bs[k]->first_slot = runs[k].first;
    bs[k]->n = runs[k].n;
    bs[k]->counts = k == 0;
  }
  if (svc->dry) {
    if (!svc->manual)
      for (int k = 0; k < m; ++k) bs[k]->complete.store(1);
  } else {
    xe_plan_t plans[xe::kMaxBatch];
    const uint8_t* gulps[xe::kMaxBatch];
    int nt[xe::kMaxBatch], acc[xe::kMaxBatch];
    for (int k = 0; k < m; ++k) {
      StreamImpl* s = who[k];
      cudaEventRecord(s->comp_mark, s->s_comp);                  // earlier correlate / integrate work
      cudaStreamWaitEvent(svc->s_batch, s->comp_mark, 0);
      cudaStreamWaitEvent(svc->s_batch, s->pending[runs[k].n - 1].h2d_done, 0);
      plans[k] = s->plan;
      gulps[k] = s->d_ring + static_cast<size_t>(runs[k].first) * s->gulp_bytes;
      nt[k] = runs[k].n * s->cfg.gulp_ntime;
      acc[k] = runs[k].accumulate ? 1 : 0;
    }
    const xe_status st = xe_correlate_batch(m, plans, gulps, nt, acc, svc->s_batch);
    if (st != XE_OK) {
      // nothing was launched: leave the runs to the single path, which
      // reports a failing launch per stream
      return;
    }
    cudaEvent_t done;
    cudaEventCreateWithFlags(&done, cudaEventDisableTiming);
    cudaEventRecord(done, svc->s_batch);
    auto* cb = new HostCbShared{{}, svc};
    for (int k = 0; k < m; ++k) {
      cudaStreamWaitEvent(who[k]->s_comp, done, 0);
      cb->b.push_back(bs[k].get());
    }
    cudaEventDestroy(done);
    if (cudaLaunchHostFunc(svc->s_batch, on_shared_done, cb) != cudaSuccess) {
      delete cb;
      for (int k = 0; k < m; ++k) fail_stream(who[k], XE_ERR_CUDA, "cudaLaunchHostFunc failed");
      return;
    }
  }
  for (int k = 0; k < m; ++k) commit_run(who[k], runs[k], std::move(bs[k]), true);
}

// The integration is complete when its last gulp has been dispatched, or on
// flush when nothing of it is pending.
void maybe_close(StreamImpl* s) {
  if (s->emit_pending || s->integ_index < 0) return;
  const int G = s->cfg.integrate_gulps;
  const long long last_of_integ = (s->integ_index + 1) * G - 1;
  bool pend_same = false;
  for (const Gulp& gp : s->pending)
    if (gp.seq / G == s->integ_index) pend_same = true;
  const bool later_seen = s->last_seq > last_of_integ;   // the writer has moved past it
  // a flush closes the integration that holds the gulps committed before it
  // (one that comes later is not affected)
  const bool flushed = s->flush_seq >= s->integ_index * G;
  if (!pend_same && (s->integ_gulps == G || later_seen || flushed)) {
    s->emit_pending = true;
    s->emit_index = s->integ_index;
  }
}

// Advance a stream as far as its state allows: close and emit finished
// integrations, dispatch pending gulps (up to kMaxInflight launches).
void pump_stream(StreamImpl* s) {
  retire(s);
  for (int guard = 0; guard < 64; ++guard) {
    bool progress = false;
    maybe_close(s);
    if (s->emit_pending) {
      if (!try_emit(s)) break;   // no free output buffer: wait for a release
      progress = true;
    }
    const size_t before = s->inflight.size();
    dispatch(s);
    if (s->inflight.size() != before) progress = true;
    if (s->svc->dry && !s->svc->manual) retire(s);   // dry-run work completes at once
    if (!progress) break;
  }
}

void pump_all(ServiceImpl* svc) {
  pump_copies(svc);
  // close and emit finished integrations first, so that their streams can
  // take part in a shared launch of the next gulps
  for (auto& s : svc->streams) {
    retire(s.get());
    maybe_close(s.get());
    if (s->emit_pending) try_emit(s.get());
  }
  if (svc->batch) dispatch_shared(svc);
  for (auto& s : svc->streams) pump_stream(s.get());
  pump_copies(svc);   // copies of integrations emitted just now
}

void worker_loop(ServiceImpl* svc) {
  std::unique_lock<std::mutex> lk(svc->mu);
  while (!svc->stop) {
    pump_all(svc);
    // with copy pieces in flight the worker polls their events more often
    const bool copying = !svc->pieces[0].empty() || !svc->pieces[1].empty();
    svc->cv.wait_for(lk, std::chrono::microseconds(copying ? 100 : 500));
  }
}

StreamImpl* get_stream(ServiceImpl* svc, int id) {
  if (id < 0 || id >= static_cast<int>(svc->streams.size())) return nullptr;
  return svc->streams[id].get();
}

void free_stream_resources(StreamImpl* s, bool dry) {
  if (dry) {
    std::free(s->h_ring);
    for (auto& p : s->h_out) std::free(p);
    return;
  }
  if (s->s_h2d) cudaStreamSynchronize(s->s_h2d);
  if (s->s_comp) cudaStreamSynchronize(s->s_comp);
  if (s->s_d2h) cudaStreamSynchronize(s->s_d2h);
  for (auto& g : s->pending)
    if (g.h2d_done) cudaEventDestroy(g.h2d_done);
  for (auto& b : s->inflight)
    if (b->done) cudaEventDestroy(b->done);
  if (s->d2h_done) cudaEventDestroy(s->d2h_done);
  if (s->comp_mark) cudaEventDestroy(s->comp_mark);
  if (s->plan) xe_plan_destroy(s->plan);
  cudaFreeHost(s->h_ring);
  for (auto& p : s->h_out) cudaFreeHost(p);
  cudaFree(s->d_ring);
  cudaFree(s->d_vis);
  if (s->s_h2d) cudaStreamDestroy(s->s_h2d);
  if (s->s_comp) cudaStreamDestroy(s->s_comp);
  if (s->s_d2h) cudaStreamDestroy(s->s_d2h);
}

}  // namespace

struct xe_service {
  ServiceImpl impl;
};

// ---------------------------------------------------------------- bounded wait
namespace xe {
namespace {
__global__ void wait_flag_kernel(const volatile int* flag, int expected, unsigned long long timeout_ns, int* status) {
  unsigned long long t0;
  asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t0));
  while (true) {
    if (*flag == expected) {
      *status = 0;
      return;
    }
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    if (t - t0 > timeout_ns) {
      *status = 1;
      return;
    }
    __nanosleep(1000);
  }
}
}  // namespace
}  // namespace xe

extern "C" {

XE_API xe_status xe_wait_flag(const int* d_flag, int expected, long long timeout_ns, int* d_status, void* stream) {
  if (!d_flag || !d_status || timeout_ns <= 0 || timeout_ns > 60000000000LL) return XE_ERR_INVALID_ARG;
  xe::wait_flag_kernel<<<1, 1, 0, static_cast<cudaStream_t>(stream)>>>(
      d_flag, expected, static_cast<unsigned long long>(timeout_ns), d_status);
  return cudaGetLastError() == cudaSuccess ? XE_OK : XE_ERR_CUDA;
}

XE_API xe_status xe_service_create(xe_service_t* out, long long mem_cap_bytes, int flags) {
  if (!out) return XE_ERR_INVALID_ARG;
  *out = nullptr;
  if (flags & ~(XE_SERVICE_DRYRUN | XE_SERVICE_MANUAL | XE_SERVICE_NO_BATCH)) return XE_ERR_INVALID_ARG;
  if ((flags & XE_SERVICE_MANUAL) && !(flags & XE_SERVICE_DRYRUN)) return XE_ERR_INVALID_ARG;
  const bool dry = flags & XE_SERVICE_DRYRUN;
  long long cap = mem_cap_bytes;
  if (cap <= 0) {
    if (dry) return XE_ERR_INVALID_ARG;
    size_t fr = 0, tot = 0;
    if (cudaMemGetInfo(&fr, &tot) != cudaSuccess) {
      cudaGetLastError();
      return XE_ERR_CUDA;
    }
    cap = static_cast<long long>(fr / 2);   // admission cap: half of the free HBM
  }
  int sms = 148;
  if (!dry) {
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess ||
        cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess || sms < 1) {
      cudaGetLastError();
      return XE_ERR_CUDA;
    }
  }
  auto* svc = new (std::nothrow) xe_service();
  if (!svc) return XE_ERR_NOMEM;
  ServiceImpl& S = svc->impl;
  S.cap = cap;
  S.num_sms = sms;
  S.batch = !(flags & XE_SERVICE_NO_BATCH);
  if (!dry && cudaStreamCreateWithFlags(&S.s_batch, cudaStreamNonBlocking) != cudaSuccess) {
    cudaGetLastError();
    delete svc;
    return XE_ERR_CUDA;
  }
  S.flags = flags;
  S.dry = dry;
  S.manual = flags & XE_SERVICE_MANUAL;
  if (!dry) S.worker = std::thread(worker_loop, &S);
  *out = svc;
  return XE_OK;
}

XE_API xe_status xe_service_destroy(xe_service_t svc) {
  if (!svc) return XE_OK;
  ServiceImpl& S = svc->impl;
  {
    std::lock_guard<std::mutex> lk(S.mu);
    S.stop = true;
  }
  S.cv.notify_all();
  if (S.worker.joinable()) S.worker.join();
  if (S.s_batch) cudaStreamSynchronize(S.s_batch);   // shared launches read every stream's ring
  for (auto& s : S.streams) free_stream_resources(s.get(), S.dry);
  for (auto& q : S.pieces)
    for (cudaEvent_t e : q) cudaEventDestroy(e);
  if (S.s_batch) cudaStreamDestroy(S.s_batch);
  delete svc;
  return XE_OK;
}

XE_API xe_status xe_service_add_stream(xe_service_t svc, const xe_stream_config* cfg, int* stream_id) {
  if (!svc || !cfg || !stream_id) return XE_ERR_INVALID_ARG;
  *stream_id = -1;
  ServiceImpl& S = svc->impl;
  const xe_stream_config c = *cfg;
  if (c.n_input < 1 || c.n_chan < 1 || c.gulp_ntime < 1 || c.ring_gulps < 1 || c.ring_gulps > 1024 ||
      c.integrate_gulps < 1 || (c.guaranteed != 0 && c.guaranteed != 1) || c.operand < 0 || c.operand > 2 ||
      c.out_type < 0 || c.out_type > 1)
    return XE_ERR_INVALID_ARG;
  if ((static_cast<long long>(c.n_chan) * c.n_input) % 16 != 0) return XE_ERR_ALIGNMENT;
  const long long max_samples = c.out_type == XE_OUT_CF32 ? XE_MAX_SAMPLES_CF32 : XE_MAX_SAMPLES_CI32;
  if (static_cast<long long>(c.integrate_gulps) * c.gulp_ntime > max_samples) return XE_ERR_ACCUM_BOUND;
  if (static_cast<long long>(c.ring_gulps) * c.gulp_ntime > (1LL << 30)) return XE_ERR_INVALID_ARG;
  auto s = std::make_unique<StreamImpl>();
  s->cfg = c;
  s->svc = &S;
  s->gulp_bytes = static_cast<size_t>(c.gulp_ntime) * c.n_chan * c.n_input;
  const long long nbl = static_cast<long long>(c.n_input) * (c.n_input + 1) / 2;
  s->vis_bytes = static_cast<size_t>(c.n_chan) * nbl * 8;
  // device: ring + plan accumulator + visibility buffer + the plan's scratch
  // for time-sliced units (sized by the device's SM count) + 1 MiB of other
  // plan memory
  s->dev_bytes = static_cast<long long>(c.ring_gulps) * s->gulp_bytes + 2LL * s->vis_bytes +
                 static_cast<long long>(xe::split_workspace_bytes(S.num_sms)) + (1LL << 20);
  s->host_bytes = static_cast<long long>(c.ring_gulps) * s->gulp_bytes + kOutSlots * static_cast<long long>(s->vis_bytes);
  std::lock_guard<std::mutex> lk(S.mu);
  if (S.used + s->dev_bytes > S.cap) {
    S.last_error = "admission: stream needs " + std::to_string(s->dev_bytes) + " device bytes, " +
                   std::to_string(S.cap - S.used) + " of the cap are left";
    return XE_ERR_NOMEM;
  }
  s->id = static_cast<int>(S.streams.size());
  s->slot_state.assign(c.ring_gulps, kFree);
  if (S.dry) {
    s->h_ring = static_cast<uint8_t*>(std::malloc(static_cast<size_t>(c.ring_gulps) * s->gulp_bytes));
    for (auto& p : s->h_out) p = std::malloc(s->vis_bytes);
    if (!s->h_ring || !s->h_out[0] || !s->h_out[1]) {
      free_stream_resources(s.get(), true);
      return XE_ERR_NOMEM;
    }
  } else {
    xe_status st = xe_plan_create(&s->plan, c.n_input, c.n_chan, c.ring_gulps * c.gulp_ntime,
                                  static_cast<xe_operand>(c.operand), static_cast<xe_out>(c.out_type));
    if (st != XE_OK) return st;
    bool ok = cudaMallocHost(&s->h_ring, static_cast<size_t>(c.ring_gulps) * s->gulp_bytes) == cudaSuccess;
    ok = ok && cudaMalloc(&s->d_ring, static_cast<size_t>(c.ring_gulps) * s->gulp_bytes) == cudaSuccess;
    ok = ok && cudaMalloc(&s->d_vis, s->vis_bytes) == cudaSuccess;
    for (auto& p : s->h_out) ok = ok && cudaMallocHost(&p, s->vis_bytes) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&s->s_h2d, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&s->s_comp, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaStreamCreateWithFlags(&s->s_d2h, cudaStreamNonBlocking) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&s->d2h_done, cudaEventDisableTiming) == cudaSuccess;
    ok = ok && cudaEventCreateWithFlags(&s->comp_mark, cudaEventDisableTiming) == cudaSuccess;
    if (ok) ok = cudaEventRecord(s->d2h_done, s->s_d2h) == cudaSuccess;
    if (!ok) {
      cudaGetLastError();
      free_stream_resources(s.get(), false);
      S.last_error = "stream allocation failed";
      return XE_ERR_NOMEM;
    }
  }
  s->st.device_bytes = s->dev_bytes;
  s->st.host_bytes = s->host_bytes;
  S.used += s->dev_bytes;
  *stream_id = s->id;
  S.streams.push_back(std::move(s));
  return XE_OK;
}

XE_API xe_status xe_service_reserve(xe_service_t svc, int id, int timeout_ms, void** h_slot) {
  if (!svc || !h_slot || timeout_ms < 0) return XE_ERR_INVALID_ARG;
  *h_slot = nullptr;
  ServiceImpl& S = svc->impl;
  std::unique_lock<std::mutex> lk(S.mu);
  StreamImpl* s = get_stream(&S, id);
  if (!s) return XE_ERR_INVALID_ARG;
  if (s->state != XE_OK) return static_cast<xe_status>(s->state);
  if (s->reserved_slot >= 0) return XE_ERR_INVALID_ARG;   // one reservation at a time
  const auto deadline = Clock::now() + std::chrono::milliseconds(s->cfg.guaranteed ? timeout_ms : 0);
  while (true) {
    pump_stream(s);
    if (s->slot_state[s->next_slot] == kFree) break;
    if (S.dry || !s->cfg.guaranteed || Clock::now() >= deadline) {
      if (!s->cfg.guaranteed) s->st.skipped_full++;
      return XE_ERR_BUSY;
    }
    S.cv.wait_until(lk, std::min(deadline, Clock::now() + std::chrono::microseconds(500)));
    if (s->state != XE_OK) return static_cast<xe_status>(s->state);
  }
  s->reserved_slot = s->next_slot;
  s->slot_state[s->next_slot] = kReserved;
  s->next_slot = (s->next_slot + 1) % s->cfg.ring_gulps;
  *h_slot = s->h_ring + static_cast<size_t>(s->reserved_slot) * s->gulp_bytes;
  return XE_OK;
}

XE_API xe_status xe_service_commit(xe_service_t svc, int id, long long seq) {
  if (!svc) return XE_ERR_INVALID_ARG;
  ServiceImpl& S = svc->impl;
  std::lock_guard<std::mutex> lk(S.mu);
  StreamImpl* s = get_stream(&S, id);
  if (!s || s->reserved_slot < 0) return XE_ERR_INVALID_ARG;
  const int slot = s->reserved_slot;
  auto unreserve = [&]() {
    // give the slot back: it is the most recently reserved one
    s->slot_state[slot] = kFree;
    s->next_slot = slot;
    s->reserved_slot = -1;
  };
  if (s->state != XE_OK) {
    unreserve();
    return static_cast<xe_status>(s->state);
  }
  if (seq <= s->last_seq || seq < 0) {   // sequence numbers increase
    unreserve();
    return XE_ERR_INVALID_ARG;
  }
  if (s->fault == XE_FAULT_DROP_GULP) {   // lost in transit: the writer moves on
    s->fault = 0;
    unreserve();
    s->last_seq = seq;
    s->st.dropped++;
    pump_stream(s);
    return XE_OK;
  }
  Gulp g{seq, slot, now_ms(), nullptr, S.dry};
  if (!S.dry) {
    if (cudaEventCreateWithFlags(&g.h2d_done, cudaEventDisableTiming) != cudaSuccess) {
      cudaGetLastError();
      unreserve();
      return fail_stream(s, XE_ERR_CUDA, "H2D copy failed");
    }
    // the copy goes out in pieces (pump_copies, below)
    const size_t off = static_cast<size_t>(slot) * s->gulp_bytes;
    auto j = std::make_unique<CopyJob>();
    j->dst = s->d_ring + off;
    j->src = s->h_ring + off;
    j->bytes = s->gulp_bytes;
    j->gulp_seq = seq;
    s->copies[0].push_back(std::move(j));
  }
  s->slot_state[slot] = kCommitted;
  s->reserved_slot = -1;
  s->last_seq = seq;
  s->st.committed++;
  s->pending.push_back(g);
  pump_all(&S);   // other streams' ready gulps may share this launch
  S.cv.notify_all();
  return XE_OK;
}

XE_API xe_status xe_service_submit(xe_service_t svc, int id, const void* h_gulp, long long seq, int timeout_ms) {
  if (!svc || !h_gulp) return XE_ERR_INVALID_ARG;
  void* slot = nullptr;
  xe_status st = xe_service_reserve(svc, id, timeout_ms, &slot);
  if (st != XE_OK) return st;
  size_t bytes;
  {
    std::lock_guard<std::mutex> lk(svc->impl.mu);
    bytes = svc->impl.streams[id]->gulp_bytes;
  }
  std::memcpy(slot, h_gulp, bytes);
  return xe_service_commit(svc, id, seq);
}

XE_API xe_status xe_service_flush(xe_service_t svc, int id) {
  if (!svc) return XE_ERR_INVALID_ARG;
  ServiceImpl& S = svc->impl;
  std::lock_guard<std::mutex> lk(S.mu);
  StreamImpl* s = get_stream(&S, id);
  if (!s) return XE_ERR_INVALID_ARG;
  s->flush_seq = s->last_seq;
  pump_stream(s);
  S.cv.notify_all();
  return XE_OK;
}

XE_API xe_status xe_service_poll(xe_service_t svc, int id, int timeout_ms, xe_integration* out) {
  if (!svc || !out || timeout_ms < 0) return XE_ERR_INVALID_ARG;
  ServiceImpl& S = svc->impl;
  std::unique_lock<std::mutex> lk(S.mu);
  StreamImpl* s = get_stream(&S, id);
  if (!s) return XE_ERR_INVALID_ARG;
  const auto deadline = Clock::now() + std::chrono::milliseconds(timeout_ms);
  while (true) {
    pump_stream(s);
    if (!s->emits.empty() && s->emits.front()->ready.load(std::memory_order_acquire)) break;
    if (S.dry || Clock::now() >= deadline) return XE_ERR_BUSY;
    S.cv.wait_until(lk, std::min(deadline, Clock::now() + std::chrono::microseconds(500)));
  }
  std::unique_ptr<Emit> e = std::move(s->emits.front());
  s->emits.pop_front();
  out->stream = id;
  out->index = e->index;
  out->first_seq = e->first_seq;
  out->gulps = e->gulps;
  out->skipped = e->skipped;
  out->samples = e->samples;
  out->latency_ms = e->t_done - e->t_last_commit;
  out->vis = s->h_out[e->out_slot];
  out->vis_bytes = static_cast<long long>(s->vis_bytes);
  out->status = e->status;
  s->handed.push_back(std::move(e));
  return XE_OK;
}

XE_API xe_status xe_service_release(xe_service_t svc, int id, long long index) {
  if (!svc) return XE_ERR_INVALID_ARG;
  ServiceImpl& S = svc->impl;
  std::lock_guard<std::mutex> lk(S.mu);
  StreamImpl* s = get_stream(&S, id);
  if (!s) return XE_ERR_INVALID_ARG;
  for (auto it = s->handed.begin(); it != s->handed.end(); ++it) {
    if ((*it)->index == index) {
      s->out_busy[(*it)->out_slot] = false;
      s->handed.erase(it);
      pump_stream(s);
      S.cv.notify_all();
      return XE_OK;
    }
  }
  return XE_ERR_INVALID_ARG;
}

XE_API xe_status xe_service_stats(xe_service_t svc, int id, xe_stream_stats* out) {
  if (!svc || !out) return XE_ERR_INVALID_ARG;
  ServiceImpl& S = svc->impl;
  std::lock_guard<std::mutex> lk(S.mu);
  StreamImpl* s = get_stream(&S, id);
  if (!s) return XE_ERR_INVALID_ARG;
  retire(s);
  *out = s->st;
  out->state = s->state;
  out->pending = static_cast<int>(s->pending.size());
  out->inflight = static_cast<int>(s->inflight.size());
  return XE_OK;
}

XE_API xe_status xe_service_inject(xe_service_t svc, int id, int fault) {
  if (!svc || (fault != XE_FAULT_LAUNCH && fault != XE_FAULT_DROP_GULP)) return XE_ERR_INVALID_ARG;
  ServiceImpl& S = svc->impl;
  std::lock_guard<std::mutex> lk(S.mu);
  StreamImpl* s = get_stream(&S, id);
  if (!s) return XE_ERR_INVALID_ARG;
  s->fault = fault;
  return XE_OK;
}

XE_API xe_status xe_service_dryrun_complete(xe_service_t svc, int id) {
  if (!svc) return XE_ERR_INVALID_ARG;
  ServiceImpl& S = svc->impl;
  if (!S.manual) return XE_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(S.mu);
  auto complete = [](StreamImpl* s) {
    for (auto& b : s->inflight) b->complete.store(1);
    for (auto& e : s->emits)
      if (!e->ready.load()) {
        e->t_done = now_ms();
        e->ready.store(1);
      }
  };
  if (id == -1) {   // every stream at once: their next runs may then share a launch
    for (auto& s : S.streams) complete(s.get());
    pump_all(&S);
    return XE_OK;
  }
  StreamImpl* s = get_stream(&S, id);
  if (!s) return XE_ERR_INVALID_ARG;
  complete(s);
  pump_stream(s);
  return XE_OK;
}

XE_API const char* xe_service_last_error(xe_service_t svc) {
  if (!svc) return "";
  std::lock_guard<std::mutex> lk(svc->impl.mu);
  thread_local std::string copy;
  copy = svc->impl.last_error;
  return copy.c_str();
}

}  // extern "C"
