// batch.cu -- batched solves of independent systems (not in the paper).
//
// A pool of host worker threads ("lanes"), each owning a handle on its own
// non-blocking stream with memory from the device pool, takes the systems
// largest first (longest-processing-time order) and runs, for each, the same
// set-up and solve as mss_setup + mss_fgmres_solve. Small systems leave most
// of the 152 SMs idle; several lanes keep them busy, and every lane's host
// synchronisations (set-up sizes, Krylov scalars) overlap with the others'
// GPU work.
//
// Autotuner: per size bucket (floor(log2 N), nb) the first system times the
// preconditioner application and the matrix-vector product at 64..512
// threads per CTA, then one solve per driver (host loop; CUDA graph with its
// capture), and caches the fastest. None of these choices changes a result.
//
// Fused schedule: the lanes only set the systems up (each on a handle of its
// own); the solves of each block size then run in lock step as one group
// through multi-system launches (fused.cu).
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cmath>
#include <map>
#include <memory>
#include <mutex>
#include <new>
#include <thread>
#include <vector>

#include "common.cuh"

using namespace mss;

namespace {

struct Choice {
  int threads = 256;
  int driver = MSS_DRIVER_HOST;
  bool ready = false;   // false while the tuning system is still running
};

using Clock = std::chrono::steady_clock;

double ms_since(Clock::time_point t0) {
  return std::chrono::duration<double, std::milli>(Clock::now() - t0).count();
}

int bucket_of(int n) {
  int b = 0;
  while ((2LL << b) <= n) ++b;
  return b;
}

// mean GPU time of `reps` runs of fn on the handle's stream, after one warm-up
template <class F>
float time_on_stream(Handle& H, int reps, F fn) {
  cudaEvent_t a, b;
  MSS_CK(cudaEventCreate(&a));
  MSS_CK(cudaEventCreate(&b));
  fn();
  MSS_CK(cudaEventRecord(a, H.stream));
  for (int r = 0; r < reps; ++r) fn();
  MSS_CK(cudaEventRecord(b, H.stream));
  MSS_CK(cudaEventSynchronize(b));
  float ms = 0.f;
  MSS_CK(cudaEventElapsedTime(&ms, a, b));
  cudaEventDestroy(a);
  cudaEventDestroy(b);
  return ms / reps;
}

}  // namespace

struct mss_batch {
  int device = 0;
  int lanes = 1;
  int autotune = 1;
  int schedule = MSS_SCHEDULE_LANES;
  FusedTuneCache fcache;        // tile shapes of the fused schedule
  // the fused schedule's per-system handles, kept between calls (the k-th
  // largest system of a call takes handle k; a set-up replaces its contents)
  std::vector<std::unique_ptr<Handle>> sysh;
  std::vector<std::unique_ptr<Handle>> grouph;   // the group solves' streams and buffers
  std::vector<std::unique_ptr<Handle>> lane;
  std::mutex mu;
  std::map<long long, Choice> cache;   // key: bucket * 16 + nb
  std::string last_error;
};

namespace {

Handle* make_lane(int device) {
  std::unique_ptr<Handle> h(new Handle());
  h->device = device;
  MSS_CK(cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, device));
  MSS_CK(cudaStreamCreateWithFlags(&h->owned.s, cudaStreamNonBlocking));
  h->stream = h->owned.s;
  mss_options_default(&h->opt);
  return h.release();
}

// Times the candidates on the set-up system in H and returns the choice;
// also leaves the system solved in sys.x (res filled).
Choice tune(Handle& H, const mss_system& s, double tol, int maxit, mss_result* res) {
  Choice c;
  const long long n = (long long)s.J.n_rows * s.nb;
  DBuf<double> r(&H, (size_t)n), y(&H, (size_t)n);
  scale_vector(&H, s.b, r.p);
  float best = 1e30f;
  for (int tb : {64, 128, 256, 512}) {
    H.tb = tb;
    const float t = time_on_stream(H, 3, [&] {
      precond_apply(&H, r.p, y.p);
      bsr_spmv(&H, y.p, r.p);
    });
    if (t < best) {
      best = t;
      c.threads = tb;
    }
  }
  H.tb = c.threads;
  double tdrv[2];
  for (int d : {MSS_DRIVER_HOST, MSS_DRIVER_GRAPH}) {
    H.opt.driver = d;
    if (H.sgraph) {   // time the graph's capture too: graphs are not shared
      cudaGraphExecDestroy(H.sgraph);
      H.sgraph = nullptr;
    }
    const auto t0 = Clock::now();
    solve_handle(H, &s.J, s.b, s.x, tol, maxit, res);
    tdrv[d] = ms_since(t0);
  }
  c.driver = tdrv[MSS_DRIVER_GRAPH] < tdrv[MSS_DRIVER_HOST] ? MSS_DRIVER_GRAPH : MSS_DRIVER_HOST;
  c.ready = true;
  return c;
}

// status code of the exception being handled (inside a catch block)
int error_code() {
  try {
    throw;
  } catch (const Error& e) {
    return e.code;
  } catch (const std::bad_alloc&) {
    return MSS_ERR_OOM;
  } catch (...) {
  }
  return MSS_ERR_CUDA;
}

void run_one(mss_batch* B, Handle& H, int lane, const mss_system& s, const mss_options& base,
             double tol, int maxit, mss_result* res, mss_batch_info* inf,
             Clock::time_point tbatch) {
  const auto t0 = Clock::now();
  mss_options o = base;
  const int bucket = bucket_of(s.J.n_rows);
  const long long key = (long long)bucket * 16 + s.nb;
  Choice c;
  bool tuner = false;
  if (B->autotune) {
    std::lock_guard<std::mutex> lk(B->mu);
    auto it = B->cache.find(key);
    if (it == B->cache.end()) {
      B->cache[key] = Choice();   // placeholder: this lane tunes the bucket
      tuner = true;
    } else if (it->second.ready) {
      c = it->second;
    }
  } else {
    c.driver = base.driver;
  }
  o.driver = c.driver;
  H.tb = c.threads;
  try {
    setup_handle(H, &s.J, s.nb, s.layout, &o);
    if (tuner) {
      c = tune(H, s, tol, maxit, res);
      std::lock_guard<std::mutex> lk(B->mu);
      B->cache[key] = c;
    } else {
      solve_handle(H, &s.J, s.b, s.x, tol, maxit, res);
    }
  } catch (...) {
    const int code = error_code();
    if (tuner) {   // let the next system of the bucket tune it
      std::lock_guard<std::mutex> lk(B->mu);
      B->cache.erase(key);
    }
    *res = mss_result{};
    res->status = code;
  }
  if (inf) {
    inf->bucket = bucket;
    inf->threads = c.threads;
    inf->driver = c.driver;
    inf->lane = lane;
    inf->latency_ms = ms_since(t0);
    inf->finish_ms = ms_since(tbatch);
    inf->schedule = MSS_SCHEDULE_LANES;
    inf->group = -1;
    inf->tile_blocks = 0;
    inf->per_sm = 0;
  }
}

// The fused schedule. The systems of each block size are split, in
// largest-first order, into kWaves groups of about equal cell counts; the
// lanes set every system up on a handle of its own (largest first), and each
// group is solved in lock step (fused_solve) on its own thread and stream as
// soon as its last set-up is done, so the group solves of the first waves
// overlap the set-ups of the later ones. The systems in `idx` are the ones it
// takes (order: largest first).
constexpr int kWaves = 3;

void batch_fused(mss_batch* B, const std::vector<int>& idx, const mss_system* sys,
                 const mss_options& base, double tol, int maxit, mss_result* results,
                 mss_batch_info* info, Clock::time_point tbatch) {
  const int n = (int)idx.size();
  if ((int)B->sysh.size() < n) B->sysh.resize((size_t)n);
  auto& hs = B->sysh;
  // groups: per nb, consecutive systems (largest first) up to 1/kWaves of the
  // nb's cells each
  std::map<int, long long> cells_of_nb;
  for (int k = 0; k < n; ++k) cells_of_nb[sys[idx[k]].nb] += sys[idx[k]].J.n_rows;
  std::vector<std::vector<int>> members;
  std::vector<int> gid((size_t)n);
  {
    std::map<int, std::pair<int, long long>> open;   // nb -> (group, cells so far)
    for (int k = 0; k < n; ++k) {
      const int nb = sys[idx[k]].nb;
      auto it = open.find(nb);
      if (it == open.end()) {
        members.emplace_back();
        it = open.emplace(nb, std::make_pair((int)members.size() - 1, 0LL)).first;
      }
      const int g = it->second.first;
      members[g].push_back(k);
      gid[k] = g;
      it->second.second += sys[idx[k]].J.n_rows;
      if (it->second.second * kWaves >= cells_of_nb[nb]) open.erase(it);   // the group is full
    }
  }
  const int ng = (int)members.size();
  if ((int)B->grouph.size() < ng) B->grouph.resize((size_t)ng);
  std::vector<double> t0((size_t)n, 0.0);
  std::vector<int> lane_of((size_t)n, 0);
  std::vector<char> ok((size_t)n, 0);
  std::vector<int> pending((size_t)ng);
  for (int g = 0; g < ng; ++g) pending[g] = (int)members[g].size();
  std::mutex mu;
  std::condition_variable cv;
  // ---- group solves: each waits for its set-ups, then runs
  auto solve_group = [&](int g) {
    cudaSetDevice(B->device);
    {
      std::unique_lock<std::mutex> lk(mu);
      cv.wait(lk, [&] { return pending[g] == 0; });
    }
    std::vector<int> ks;
    for (int k : members[g])
      if (ok[k]) ks.push_back(k);
    if (ks.empty()) return;
    std::vector<Handle*> hv;
    std::vector<const double*> bv;
    std::vector<double*> xv;
    for (int k : ks) {
      hv.push_back(hs[k].get());
      bv.push_back(sys[idx[k]].b);
      xv.push_back(sys[idx[k]].x);
    }
    std::vector<mss_result> res;
    FusedInfo fi;
    int code = MSS_OK;
    const auto ts = Clock::now();
    try {
      if (!B->grouph[g]) B->grouph[g].reset(make_lane(B->device));
      Handle* gh = B->grouph[g].get();
      fused_solve(gh, hv, bv, xv, tol, maxit, base.driver, B->autotune ? &B->fcache : nullptr,
                  res, &fi);
      MSS_CK(cudaStreamSynchronize(gh->stream));
    } catch (...) {
      code = error_code();
    }
    const double solve_ms = ms_since(ts), tend = ms_since(tbatch);
    for (size_t q = 0; q < ks.size(); ++q) {
      const int k = ks[q], i = idx[k];
      if (code == MSS_OK) {
        results[i] = res[q];
        results[i].solve_ms = solve_ms;
      } else {
        results[i] = mss_result{};
        results[i].status = code;
      }
      if (info) {
        mss_batch_info& f = info[i];
        f.bucket = bucket_of(sys[i].J.n_rows);
        f.threads = 256;
        f.driver = base.driver;
        f.lane = lane_of[k];
        f.latency_ms = tend - t0[k];
        f.finish_ms = tend;
        f.schedule = MSS_SCHEDULE_FUSED;
        f.group = g;
        f.tile_blocks = fi.tile_blocks;
        f.per_sm = fi.per_sm;
      }
    }
  };
  std::vector<std::thread> gt;
  for (int g = 0; g < ng; ++g) gt.emplace_back(solve_group, g);
  // ---- set-ups on the lanes, largest first
  std::atomic<int> next{0};
  auto work = [&](int l) {
    cudaSetDevice(B->device);
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= n) break;
      const int i = idx[k];
      t0[k] = ms_since(tbatch);
      lane_of[k] = l;
      try {
        if (!hs[k]) hs[k].reset(make_lane(B->device));
        setup_handle(*hs[k], &sys[i].J, sys[i].nb, sys[i].layout, &base);
        MSS_CK(cudaStreamSynchronize(hs[k]->stream));
        ok[k] = 1;
      } catch (...) {
        results[i] = mss_result{};
        results[i].status = error_code();
      }
      {
        std::lock_guard<std::mutex> lk(mu);
        --pending[gid[k]];
      }
      cv.notify_all();
    }
  };
  {
    const int nl = std::min(B->lanes, n);
    std::vector<std::thread> th;
    for (int l = 1; l < nl; ++l) th.emplace_back(work, l);
    work(0);
    for (auto& t : th) t.join();
  }
  for (auto& t : gt) t.join();
  for (int k = 0; k < n; ++k)
    if (hs[k]) cudaStreamSynchronize(hs[k]->stream);
}

}  // namespace

extern "C" {

int mss_batch_create(mss_batch** out, int lanes, int autotune) {
  if (!out || lanes < 1 || lanes > 64) return MSS_ERR_INVALID_ARG;
  *out = nullptr;
  mss_batch* B = new (std::nothrow) mss_batch();
  if (!B) return MSS_ERR_OOM;
  try {
    MSS_CK(cudaGetDevice(&B->device));
    B->lanes = lanes;
    B->autotune = autotune != 0;
    for (int i = 0; i < lanes; ++i) B->lane.emplace_back(make_lane(B->device));
  } catch (const Error& e) {
    delete B;
    return e.code;
  } catch (...) {
    delete B;
    return MSS_ERR_OOM;
  }
  *out = B;
  return MSS_OK;
}

void mss_batch_destroy(mss_batch* B) {
  if (!B) return;
  for (auto& h : B->lane)
    if (h) cudaStreamSynchronize(h->stream);
  for (auto& h : B->sysh)
    if (h) cudaStreamSynchronize(h->stream);
  for (auto& h : B->grouph)
    if (h) cudaStreamSynchronize(h->stream);
  delete B;
  trim_pools();
}

int mss_batch_solve(mss_batch* B, int n, const mss_system* sys, const mss_options* opt,
                    double tol, int maxit, mss_result* results, mss_batch_info* info) {
  if (!B) return MSS_ERR_INVALID_ARG;
  if (n < 0 || (n > 0 && (!sys || !results)) || !(tol >= 0.0) || maxit < 0) {
    B->last_error = "bad batch arguments";
    return MSS_ERR_INVALID_ARG;
  }
  if (n == 0) return MSS_OK;
  mss_options base;
  if (opt) base = *opt;
  else mss_options_default(&base);
  if (cudaSetDevice(B->device) != cudaSuccess || cudaDeviceSynchronize() != cudaSuccess) {
    cudaGetLastError();
    B->last_error = "device synchronisation failed";
    return MSS_ERR_CUDA;
  }
  // largest first: block-row work nnzb * nb^2
  std::vector<int> order(n);
  for (int i = 0; i < n; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int a, int b) {
    const double wa = (double)sys[a].J.nnzb * sys[a].nb * sys[a].nb;
    const double wb = (double)sys[b].J.nnzb * sys[b].nb * sys[b].nb;
    return wa > wb;
  });
  const auto tbatch = Clock::now();
  if (B->schedule == MSS_SCHEDULE_FUSED && fused_supported(base, kFusedMaxNB)) {
    // systems of nb <= kFusedMaxNB take the fused schedule, the others the lanes
    std::vector<int> fused, rest;
    for (int i : order) (sys[i].nb <= kFusedMaxNB ? fused : rest).push_back(i);
    batch_fused(B, fused, sys, base, tol, maxit, results, info, tbatch);
    order = rest;
  }
  std::atomic<int> next{0};
  const int nrest = (int)order.size();
  auto work = [&](int l) {
    cudaSetDevice(B->device);
    Handle& H = *B->lane[l];
    for (;;) {
      const int k = next.fetch_add(1);
      if (k >= nrest) break;
      const int i = order[k];
      run_one(B, H, l, sys[i], base, tol, maxit, &results[i], info ? &info[i] : nullptr,
              tbatch);
    }
  };
  if (nrest > 0) {
    const int nl = std::min(B->lanes, nrest);
    std::vector<std::thread> th;
    for (int l = 1; l < nl; ++l) th.emplace_back(work, l);
    work(0);
    for (auto& t : th) t.join();
  }
  int st = MSS_OK;
  for (int i = 0; i < n && st == MSS_OK; ++i) st = results[i].status;
  B->last_error = st == MSS_OK ? "" : "a system did not converge or failed; see its result";
  return st;
}

int mss_batch_set_schedule(mss_batch* B, int schedule) {
  if (!B || (schedule != MSS_SCHEDULE_LANES && schedule != MSS_SCHEDULE_FUSED))
    return MSS_ERR_INVALID_ARG;
  B->schedule = schedule;
  return MSS_OK;
}

int mss_batch_tuned(mss_batch* B, int cap, int32_t* out) {
  if (!B || cap < 0 || (cap > 0 && !out)) return MSS_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lk(B->mu);
  int k = 0;
  for (auto& kv : B->cache) {
    if (!kv.second.ready) continue;
    if (k < cap) {
      out[4 * k + 0] = (int32_t)(kv.first / 16);
      out[4 * k + 1] = (int32_t)(kv.first % 16);
      out[4 * k + 2] = kv.second.threads;
      out[4 * k + 3] = kv.second.driver;
    }
    ++k;
  }
  return k;
}

const char* mss_batch_last_error(const mss_batch* B) {
  return B ? B->last_error.c_str() : "null batch";
}

}  // extern "C"
