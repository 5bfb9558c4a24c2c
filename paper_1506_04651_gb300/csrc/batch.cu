// Batched serving: many independent instances (each its own grid, depth,
// parameters and threshold) stepped together on one GPU.  Every instance
// keeps its own context and CUDA stream; the grid adaptation of all
// instances runs concurrently, driven by a pool of host threads (its phases
// synchronise with the host to size the trees).  The two reaction sub-steps
// of every Strang step run as one persistent Radau5 launch over the union of
// all instances' leaves, so that the stiff cells of one instance overlap the
// cells at rest of the others and the launch has one tail instead of one per
// instance; the diffusion sub-step runs as one persistent ROCK4 launch over
// all instances (each with its own step control), so that the grid-wide
// barriers of the stages are paid once for the batch, not once per instance.
#include <math.h>
#include <string.h>

#include <algorithm>
#include <chrono>
#include <atomic>
#include <condition_variable>
#include <functional>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "mr_internal.cuh"
#include "radau_common.cuh"

namespace mrg {
namespace {

// fixed pool of host threads running f(0 .. n-1) on demand
class Pool {
 public:
  Pool(int nthreads, int dev) : dev_(dev) {
    for (int q = 0; q < nthreads; q++) th_.emplace_back([this] { worker(); });
  }
  ~Pool() {
    {
      std::lock_guard<std::mutex> lk(mu_);
      stop_ = true;
    }
    cv_.notify_all();
    for (auto& t : th_) t.join();
  }
  void run(int n, const std::function<void(int)>& f) {
    std::unique_lock<std::mutex> lk(mu_);
    f_ = &f;
    n_ = n;
    next_ = 0;
    busy_ = (int)th_.size();
    gen_++;
    cv_.notify_all();
    done_.wait(lk, [this] { return busy_ == 0; });
    f_ = nullptr;
  }

 private:
  void worker() {
    cudaSetDevice(dev_);
    int seen = 0;
    for (;;) {
      const std::function<void(int)>* f;
      int n;
      {
        std::unique_lock<std::mutex> lk(mu_);
        cv_.wait(lk, [&] { return stop_ || gen_ != seen; });
        if (stop_) return;
        seen = gen_;
        f = f_;
        n = n_;
      }
      for (int i = next_++; i < n; i = next_++) (*f)(i);
      std::lock_guard<std::mutex> lk(mu_);
      if (--busy_ == 0) done_.notify_all();
    }
  }
  std::vector<std::thread> th_;
  std::mutex mu_;
  std::condition_variable cv_, done_;
  const std::function<void(int)>* f_ = nullptr;
  int n_ = 0, gen_ = 0, busy_ = 0;
  std::atomic<int> next_{0};
  bool stop_ = false;
  int dev_;
};

// Online autotuner of one joint launch: its candidate launch shapes are
// tried in turn on the first real launches, each for `reps` consecutive
// launches, ranked by algorithmic work per millisecond of device time (the
// launches differ in their work, so the rate, not the time, is compared),
// and the fastest is kept from then on.  The reaction's two half steps of a
// Strang step differ systematically (after the adaptation, after the
// diffusion), so with reps = 2 every candidate sees one of each.  Only shapes
// that leave the results unchanged are candidates, so tuning never changes
// what a run computes.
struct Tuner {
  struct Cand {
    int a, b;   // the shape: (threads per block, queue order) or (blocks per SM, 0)
    int c = 0;  // Radau5 schedule (MR_RADAU_THREAD or MR_RADAU_POOL)
    int64_t launches = 0;
    double ms = 0.0, work = 0.0;
  };
  std::vector<Cand> cand;
  int reps = 2, chosen = -1, next = 0;
  bool on = true;
  // the candidate for the next launch
  int pick() {
    if (!on) return 0;
    if (chosen >= 0) return chosen;
    return (next / reps) % (int)cand.size();
  }
  void record(int k, double ms, double work) {
    Cand& c = cand[k];
    c.launches++;
    c.ms += ms;
    c.work += work;
    if (!on || chosen >= 0) return;
    next++;
    if (next >= (int)cand.size() * reps) {
      double best = -1.0;
      for (int q = 0; q < (int)cand.size(); q++) {
        const double rate = cand[q].ms > 0.0 ? cand[q].work / cand[q].ms : 0.0;
        if (rate > best) {
          best = rate;
          chosen = q;
        }
      }
    }
  }
};

}  // namespace
}  // namespace mrg

struct mr_batch {
  int n = 0, dev = 0;
  std::vector<mr_ctx*> ctx;
  std::vector<cudaStream_t> streams;
  std::vector<cudaEvent_t> ev;  // one per instance
  cudaStream_t stream = nullptr;
  cudaEvent_t ev_start = nullptr, ev_end = nullptr, ev_joint = nullptr;
  mrg::Pool* pool = nullptr;
  mrg::BatchReactScratch scratch;
  mrg::BatchRockScratch rscratch;
  // the joint Radau5 launch: the thread schedule with 128 or 64 threads
  // per block, or the pooled schedule, each with the finest levels first or
  // in leaf order (the default first); the joint ROCK4 launch: 2 or 1 blocks
  // per SM
  mrg::Tuner tune_react{{{128, 1, MR_RADAU_THREAD},
                         {64, 1, MR_RADAU_THREAD},
                         {128, 0, MR_RADAU_THREAD},
                         {64, 0, MR_RADAU_THREAD},
                         {128, 1, MR_RADAU_POOL},
                         {128, 0, MR_RADAU_POOL}}};
  mrg::Tuner tune_diffuse{{{2, 0}, {1, 0}}};
  mr_batch_stats stats;
  const char* last_error = "";
};

using namespace mrg;

namespace {

void batch_free(mr_batch* b) {
  delete b->pool;
  for (mr_ctx* c : b->ctx)
    if (c) mr_destroy(c);
  for (cudaStream_t s : b->streams)
    if (s) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->ev)
    if (e) cudaEventDestroy(e);
  if (b->ev_start) cudaEventDestroy(b->ev_start);
  if (b->ev_end) cudaEventDestroy(b->ev_end);
  if (b->ev_joint) cudaEventDestroy(b->ev_joint);
  if (b->stream) cudaStreamDestroy(b->stream);
  free_batch_scratch(b->scratch);
  free_batch_rock(b->rscratch);
  delete b;
}

// run f on every instance with the pool; the first error wins
mr_status for_all(mr_batch* b, const std::function<mr_status(int)>& f) {
  std::atomic<int> first{0};
  std::function<void(int)> g = [&](int i) {
    const mr_status s = f(i);
    if (s) {
      int z = 0;
      first.compare_exchange_strong(z, (int)s);
    }
  };
  b->pool->run(b->n, g);
  return (mr_status)first.load();
}

// both reaction half steps: one joint launch when every instance uses a
// one-thread-per-cell model with the same precision, else per instance
mr_status react_all(mr_batch* b, double dt, double rtol, double atol) {
  bool joint = true;
  for (mr_ctx* c : b->ctx)
    joint = joint && (c->prob.model == MR_MODEL_BZ || c->prob.model == MR_MODEL_NAGUMO) &&
            c->prob.model == b->ctx[0]->prob.model && c->prob.precision == b->ctx[0]->prob.precision;
  if (!joint) {
    b->stats.joint_reaction = 0;
    return for_all(b, [&](int i) { return react(b->ctx[i], dt, rtol, atol); });
  }
  // the joint launch follows every instance's queued work and precedes its next
  for (int i = 0; i < b->n; i++) {
    if (cudaEventRecord(b->ev[i], b->streams[i]) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->ev[i], 0) != cudaSuccess)
      return MR_ECUDA;
  }
  double ms = 0.0;
  unsigned long long cnt[7] = {0, 0, 0, 0, 0, 0, 0};
  const int k = b->tune_react.pick();
  RadauShape shape;
  shape.block = b->tune_react.cand[k].a;
  shape.rev = b->tune_react.cand[k].b;
  shape.pool = b->tune_react.cand[k].c == MR_RADAU_POOL;
  const mr_status s = react_batch(b->ctx.data(), b->n, dt, rtol, atol, b->stream, b->scratch, &ms, cnt, shape);
  if (s) return s;
  if (cudaEventRecord(b->ev_joint, b->stream) != cudaSuccess) return MR_ECUDA;
  for (int i = 0; i < b->n; i++)
    if (cudaStreamWaitEvent(b->streams[i], b->ev_joint, 0) != cudaSuccess) return MR_ECUDA;
  mr_batch_stats& S = b->stats;
  S.joint_reaction = 1;
  S.ms_react_kernel += ms;
  S.react_launches++;
  S.radau_fev += cnt[0];
  S.radau_jac += cnt[1];
  S.radau_steps += cnt[2];
  S.radau_accept += cnt[3];
  S.radau_reject += cnt[4];
  S.radau_newton += cnt[5];
  S.radau_dec += cnt[6];
  // algorithmic FP64 operations (radau_work: counted from the kernel's source)
  int64_t cells = 0;
  for (mr_ctx* c : b->ctx) cells += c->tb[c->cur].nleaves;
  const double work = radau_alg_flops(radau_work(b->ctx[0]->prob.model, b->ctx[0]->m), cnt, cells);
  S.radau_alg_flops += work;
  b->tune_react.record(k, ms, work);
  return MR_OK;
}

// the diffusion sub-step: one joint launch when every instance is 2D with
// one or three species, all alike in species count and precision, else
// per instance (concurrently)
mr_status diffuse_all(mr_batch* b, double dt, double tol) {
  const mr_ctx* c0 = b->ctx[0];
  bool joint = c0->d == 2 && (c0->m == 1 || c0->m == 3) && b->n * c0->m <= 512;
  for (mr_ctx* c : b->ctx) joint = joint && c->d == 2 && c->m == c0->m && c->prob.precision == c0->prob.precision;
  if (!joint) {
    b->stats.joint_diffusion = 0;
    return for_all(b, [&](int i) { return diffuse(b->ctx[i], dt, tol); });
  }
  for (int i = 0; i < b->n; i++) {
    if (cudaEventRecord(b->ev[i], b->streams[i]) != cudaSuccess ||
        cudaStreamWaitEvent(b->stream, b->ev[i], 0) != cudaSuccess)
      return MR_ECUDA;
  }
  double ms = 0.0, bytes0 = 0.0, bytes1 = 0.0;
  for (mr_ctx* c : b->ctx) bytes0 += c->stats.rock_alg_bytes;
  const int k = b->tune_diffuse.pick();
  const mr_status s =
      diffuse_batch(b->ctx.data(), b->n, dt, tol, b->stream, b->rscratch, &ms, b->tune_diffuse.cand[k].a);
  if (s) return s;
  for (mr_ctx* c : b->ctx) bytes1 += c->stats.rock_alg_bytes;
  b->tune_diffuse.record(k, ms, bytes1 - bytes0);
  if (cudaEventRecord(b->ev_joint, b->stream) != cudaSuccess) return MR_ECUDA;
  for (int i = 0; i < b->n; i++)
    if (cudaStreamWaitEvent(b->streams[i], b->ev_joint, 0) != cudaSuccess) return MR_ECUDA;
  b->stats.joint_diffusion = 1;
  b->stats.ms_diffuse_kernel += ms;
  b->stats.diffuse_launches++;
  return MR_OK;
}

void reset_counters(mr_batch_stats& S) {
  S.steps = 0;
  S.leaf_updates = 0;
  S.ms_react_kernel = 0.0;
  S.react_launches = 0;
  S.radau_fev = S.radau_jac = S.radau_steps = S.radau_accept = S.radau_reject = S.radau_newton = S.radau_dec = 0;
  S.radau_alg_flops = 0.0;
  S.ms_adapt_phase = S.ms_diffuse_phase = S.ms_diffuse_kernel = 0.0;
  S.diffuse_launches = 0;
}

}  // namespace

extern "C" {

mr_status mr_batch_create(int n, const mr_problem* probs, int threads, mr_batch** out) {
  if (!out || !probs || n < 1 || n > 4096) return MR_EINVAL;
  *out = nullptr;
  mr_batch* b = new (std::nothrow) mr_batch();
  if (!b) return MR_ENOMEM;
  memset(&b->stats, 0, sizeof b->stats);
  b->n = n;
  cudaGetDevice(&b->dev);
  b->ctx.assign(n, nullptr);
  b->streams.assign(n, nullptr);
  b->ev.assign(n, nullptr);
  mr_status s = MR_OK;
  if (cudaStreamCreateWithFlags(&b->stream, cudaStreamNonBlocking) != cudaSuccess ||
      cudaEventCreate(&b->ev_start) != cudaSuccess || cudaEventCreate(&b->ev_end) != cudaSuccess ||
      cudaEventCreateWithFlags(&b->ev_joint, cudaEventDisableTiming) != cudaSuccess)
    s = MR_ECUDA;
  for (int i = 0; i < n && !s; i++) {
    if (cudaStreamCreateWithFlags(&b->streams[i], cudaStreamNonBlocking) != cudaSuccess ||
        cudaEventCreateWithFlags(&b->ev[i], cudaEventDisableTiming) != cudaSuccess) {
      s = MR_ECUDA;
      break;
    }
    s = mr_create(&probs[i], b->streams[i], &b->ctx[i]);
  }
  if (s) {
    batch_free(b);
    return s;
  }
  const int hw = (int)std::max(1u, std::thread::hardware_concurrency());
  const int nt = std::max(1, std::min(n, threads > 0 ? threads : std::min(hw, 32)));
  b->pool = new (std::nothrow) Pool(nt, b->dev);
  if (!b->pool) {
    batch_free(b);
    return MR_ENOMEM;
  }
  b->stats.instances = n;
  b->stats.threads = nt;
  *out = b;
  return MR_OK;
}

mr_ctx* mr_batch_context(mr_batch* b, int i) { return (b && i >= 0 && i < b->n) ? b->ctx[i] : nullptr; }

mr_status mr_batch_run(mr_batch* b, int nsteps, double dt, const double* eta, double rtol, double atol,
                       double rock_tol) {
  if (!b || nsteps < 0 || !eta || !(dt > 0.0) || !(rtol > 0.0) || !(atol > 0.0) || !(rock_tol > 0.0))
    return MR_EINVAL;
  for (int i = 0; i < b->n; i++)
    if (!(eta[i] >= 0.0) || !isfinite(eta[i])) return MR_EINVAL;
  mr_batch_stats& S = b->stats;
  reset_counters(S);
  using clk = std::chrono::steady_clock;
  auto ms_since = [](clk::time_point t0) {
    return std::chrono::duration<double, std::milli>(clk::now() - t0).count();
  };
  // device time from the start event (which every instance stream waits on)
  // to the end event (which waits on every instance stream)
  if (cudaEventRecord(b->ev_start, b->stream) != cudaSuccess) return MR_ECUDA;
  for (int i = 0; i < b->n; i++)
    if (cudaStreamWaitEvent(b->streams[i], b->ev_start, 0) != cudaSuccess) return MR_ECUDA;
  mr_status s = MR_OK;
  for (int step = 0; step < nsteps && !s; step++) {
    clk::time_point t0 = clk::now();
    s = for_all(b, [&](int i) {
      mr_status r = adapt(b->ctx[i], eta[i]);
      return r ? r : build_tables(b->ctx[i]);
    });
    S.ms_adapt_phase += ms_since(t0);
    if (s) break;
    for (mr_ctx* c : b->ctx) S.leaf_updates += c->tb[c->cur].nleaves;
    s = react_all(b, 0.5 * dt, rtol, atol);
    if (s) break;
    t0 = clk::now();
    s = diffuse_all(b, dt, rock_tol);
    S.ms_diffuse_phase += ms_since(t0);
    if (s) break;
    s = react_all(b, 0.5 * dt, rtol, atol);
    S.steps++;
  }
  for (int i = 0; i < b->n; i++) {
    cudaEventRecord(b->ev[i], b->streams[i]);
    cudaStreamWaitEvent(b->stream, b->ev[i], 0);
  }
  cudaEventRecord(b->ev_end, b->stream);
  if (cudaEventSynchronize(b->ev_end) != cudaSuccess && !s) s = MR_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev_start, b->ev_end);
  S.ms_device = ms;
  if (s) b->last_error = "a batched step failed (see the instance contexts' last errors)";
  return s;
}

mr_status mr_batch_diffuse(mr_batch* b, double dt, double tol) {
  if (!b || !(dt > 0.0) || !isfinite(dt) || !(tol > 0.0)) return MR_EINVAL;
  reset_counters(b->stats);
  if (cudaEventRecord(b->ev_start, b->stream) != cudaSuccess) return MR_ECUDA;
  for (int i = 0; i < b->n; i++)
    if (cudaStreamWaitEvent(b->streams[i], b->ev_start, 0) != cudaSuccess) return MR_ECUDA;
  mr_status s = for_all(b, [&](int i) { return build_tables(b->ctx[i]); });
  const auto t0 = std::chrono::steady_clock::now();
  if (!s) s = diffuse_all(b, dt, tol);
  b->stats.ms_diffuse_phase =
      std::chrono::duration<double, std::milli>(std::chrono::steady_clock::now() - t0).count();
  for (int i = 0; i < b->n; i++) {
    cudaEventRecord(b->ev[i], b->streams[i]);
    cudaStreamWaitEvent(b->stream, b->ev[i], 0);
  }
  cudaEventRecord(b->ev_end, b->stream);
  if (cudaEventSynchronize(b->ev_end) != cudaSuccess && !s) s = MR_ECUDA;
  float ms = 0.f;
  cudaEventElapsedTime(&ms, b->ev_start, b->ev_end);
  b->stats.ms_device = ms;
  if (s) b->last_error = "a batched diffusion failed (see the instance contexts' last errors)";
  return s;
}

mr_status mr_batch_get_stats(const mr_batch* b, mr_batch_stats* out) {
  if (!b || !out) return MR_EINVAL;
  *out = b->stats;
  return MR_OK;
}

mr_status mr_batch_set_autotune(mr_batch* b, int on) {
  if (!b || (on != 0 && on != 1)) return MR_EINVAL;
  for (Tuner* t : {&b->tune_react, &b->tune_diffuse}) {
    t->on = on != 0;
    t->chosen = on ? -1 : 0;
    t->next = 0;
    for (Tuner::Cand& c : t->cand) c = Tuner::Cand{c.a, c.b, c.c};
  }
  return MR_OK;
}

mr_status mr_batch_tuning(const mr_batch* b, mr_tune_entry* out, int cap, int* n) {
  if (!b || !n || cap < 0 || (cap > 0 && !out)) return MR_EINVAL;
  int k = 0;
  const Tuner* ts[2] = {&b->tune_react, &b->tune_diffuse};
  for (int phase = 0; phase < 2; phase++)
    for (int q = 0; q < (int)ts[phase]->cand.size(); q++, k++) {
      if (k >= cap) continue;
      const Tuner::Cand& c = ts[phase]->cand[q];
      mr_tune_entry& e = out[k];
      memset(&e, 0, sizeof e);
      e.phase = phase;
      e.block = phase == 0 ? c.a : 256;
      e.per_sm = phase == 0 ? 0 : c.a;
      e.order = phase == 0 ? c.b : 0;
      e.launches = c.launches;
      e.ms = c.ms;
      e.work = c.work;
      e.rate = c.ms > 0.0 ? c.work / c.ms : 0.0;
      e.chosen = ts[phase]->chosen == q;
      e.schedule = phase == 0 ? c.c : 0;
    }
  *n = k;
  return k > cap ? MR_ENOMEM : MR_OK;
}

void mr_batch_destroy(mr_batch* b) {
  if (b) batch_free(b);
}

}  // extern "C"
