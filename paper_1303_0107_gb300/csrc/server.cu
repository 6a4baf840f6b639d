// Request loop with continuous batching (the serving entry points of
// include/lbm.h).  Host code only.
//
// One scheduler thread owns a persistent engine whose member list is the set
// of resident requests.  Each tick it
//   1. admits queued requests in arrival order while a slot is free and the
//      summed footprint of the resident requests stays within the budget
//      (allocation, upload and initial state of Sec. 3.3 per request);
//   2. rebuilds the engine's layout and work-list if the list changed;
//   3. runs the exchange of Sec. 2.3 steps 3-4 for the requests that start an
//      optimiser iteration (one launch sequence over just those members);
//   4. advances every resident request by S time steps in the same launches,
//      S = min(max_tick_steps, the fewest steps any request has left in its
//      current solve), so every solve ends exactly at a tick boundary, where
//      the moments of its last step and its FP64 reductions are taken;
//   5. retires the requests whose last solve ended.
// A request's populations, mask and fields stay on the device from
// admission to retirement.  The kernels compute every cell and every
// reduction of a member from that member's data alone, in an order fixed by
// the member, so a request's results do not depend on what else is resident.
#include <algorithm>
#include <chrono>
#include <set>
#include <cmath>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <vector>

#include "engine.h"

using namespace lbm;

namespace {

struct Pending {
  lbm_request r{};
  std::vector<uint8_t> cells;
  double t_submit = 0.0;
  int64_t footprint = 0;
};

struct Slot {
  Pending q;
  Member* m = nullptr;
  double t_admit = 0.0;
  int iter = 0;              // optimiser iterations started
  int64_t steps_left = 0;    // in the current solve
  bool exchange_next = false;
  bool first_done = false;
  int32_t n_swapped = 0;
  int64_t fluid_updates = 0;
  double dp_first = NAN;
  lbm_solve_result last{};
};

// one engine indexes the cells of its members with 32-bit integers
constexpr int64_t kMaxSetCells = (int64_t)1 << 31;

int64_t cells_of(const Pending& p) { return (int64_t)p.r.params.nx * p.r.params.ny; }

int64_t footprint_of(const lbm_params& p, int32_t n_iter) {
  const int64_t cells = (int64_t)p.nx * p.ny;
  // the member's own allocation; its share of the set's work-list (segment
  // entries with their neighbour flags, 72 bytes per 32-cell word, and scan
  // scratch: under 3 bytes per cell), of the compacted cell list the request
  // loop steps (an 8-byte entry per fluid cell, and its scan scratch: under
  // 9 bytes per cell) and of the read-back buffer (4 bytes per cell); for
  // optimising requests the exchange scratch: counts and offsets per mask
  // word, 24 bytes of keys and indices per cell and 4 bytes of picks per cell
  int64_t b = (int64_t)member_footprint(p) + 16 * cells + 4096;
  if (n_iter > 0) b += 29 * cells;
  return b;
}

size_t engine_buffer_bytes(const Engine* E) {
  size_t b = 0;
  for (const GrowBuf* g : {&E->L.views, &E->L.word_off, &E->L.seg_word_off, &E->XL.views, &E->XL.word_off,
                           &E->XL.seg_word_off, &E->segs, &E->n_segs, &E->seg_scratch, &E->partials, &E->result,
                           &E->fluid_dev, &E->n_swap_dev, &E->dense_f, &E->oc_buf, &E->bar})
    b += g->cap;
  return b;
}

}  // namespace

struct lbm_server_s {
  lbm_server_config cfg{};
  int64_t budget = 0;
  int device = 0;
  Engine* E = nullptr;
  std::chrono::steady_clock::time_point t0;

  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Pending> queue;   // guarded by mu
  std::deque<lbm_served> done; // guarded by mu
  int64_t resident = 0;        // guarded by mu
  int64_t resident_cells = 0;  // guarded by mu
  lbm_server_stats st{};       // guarded by mu
  std::set<int64_t> cancel;    // tags of resident requests to withdraw; guarded by mu
  std::set<int64_t> resident_tags;  // guarded by mu
  bool stop = false;           // guarded by mu
  bool fatal = false;          // guarded by mu
  std::vector<Slot> slots;     // scheduler thread only
  std::thread th;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }

  void finish(Slot& s, int32_t status) {
    lbm_served d;
    std::memset(&d, 0, sizeof(d));
    d.tag = s.q.r.tag;
    d.status = status;
    d.n_swapped = s.n_swapped;
    d.t_submit = s.q.t_submit;
    d.t_admit = s.t_admit;
    d.t_done = now();
    d.fluid_updates = s.fluid_updates;
    d.footprint_bytes = s.q.footprint;
    d.dp_first = s.dp_first;
    d.last = s.last;
    std::lock_guard<std::mutex> lk(mu);
    done.push_back(d);
    resident -= s.q.footprint;
    st.resident_bytes = resident;
    resident_tags.erase(s.q.r.tag);
    cancel.erase(s.q.r.tag);
    resident_cells -= cells_of(s.q);
    if (status == LBM_OK) ++st.completed; else ++st.failed;
    cv_done.notify_all();
  }

  void finish_pending(Pending& p, int32_t status, double t) {
    Slot s;
    s.q = std::move(p);
    s.t_admit = t;
    finish(s, status);
  }

  // A CUDA failure leaves the stream unusable: fail everything and stop.
  void fail_all(int32_t status) {
    for (Slot& s : slots) {
      finish(s, status);
      delete s.m;
    }
    slots.clear();
    std::deque<Pending> q;
    {
      std::lock_guard<std::mutex> lk(mu);
      fatal = true;
      q.swap(queue);
      for (const Pending& p : q) {  // finish() releases what admission would have charged
        resident += p.footprint;
        resident_cells += cells_of(p);
      }
    }
    for (Pending& p : q) finish_pending(p, status, now());
  }

  void loop();
};

void lbm_server_s::loop() {
  cudaSetDevice(device);
  bool changed = false;
  for (;;) {
    std::vector<Pending> adm;
    {
      std::unique_lock<std::mutex> lk(mu);
      cv_work.wait(lk, [&] { return stop || !queue.empty() || !slots.empty(); });
      if (stop) return;
      while (!queue.empty() && (int)(slots.size() + adm.size()) < cfg.max_active &&
             resident + queue.front().footprint <= budget &&
             resident_cells + cells_of(queue.front()) < kMaxSetCells) {
        resident += queue.front().footprint;
        resident_cells += cells_of(queue.front());
        resident_tags.insert(queue.front().r.tag);
        adm.push_back(std::move(queue.front()));
        queue.pop_front();
      }
      st.admitted += (int64_t)adm.size();
      st.queued = (int32_t)queue.size();
      st.resident_bytes = resident;
      st.peak_resident_bytes = std::max(st.peak_resident_bytes, resident);
    }
    NvtxRange nvtx("lbm_server_tick");  // admission, exchange, steps, retirement
    const double t_tick = now();
    for (Pending& p : adm) {
      Member* m = nullptr;
      lbm_status s = member_create(p.r.params, p.cells.data(), E->stream, &m);
      if (s == LBM_OK) s = member_reset(m, E->stream);
      if (s != LBM_OK) {
        delete m;
        finish_pending(p, s, t_tick);
        continue;
      }
      Slot sl;
      sl.q = std::move(p);
      sl.q.cells = std::vector<uint8_t>();  // on the device from here on
      sl.m = m;
      sl.t_admit = t_tick;
      sl.steps_left = sl.q.r.n_steps;
      slots.push_back(std::move(sl));
      changed = true;
    }
    bool withdrew = false;
    {  // withdraw cancelled resident requests before this tick
      std::vector<int64_t> gone;
      {
        std::lock_guard<std::mutex> lk(mu);
        gone.assign(cancel.begin(), cancel.end());
      }
      if (!gone.empty()) {
        std::vector<Slot> keep;
        for (Slot& x : slots) {
          if (std::find(gone.begin(), gone.end(), x.q.r.tag) != gone.end()) {
            finish(x, LBM_ERR_CANCELLED);
            delete x.m;
            changed = true;
            withdrew = true;
          } else {
            keep.push_back(std::move(x));
          }
        }
        slots.swap(keep);
        if (slots.empty()) E->m.clear();
      }
    }
    if (slots.empty()) {
      // a withdrawal freed room after this tick's admission: admit again first
      if (withdrew) continue;
      // nothing resident and nothing admitted (only if a request can never fit)
      std::unique_lock<std::mutex> lk(mu);
      if (!queue.empty() && adm.empty()) {
        Pending p = std::move(queue.front());
        queue.pop_front();
        resident += p.footprint;
        resident_cells += cells_of(p);
        lk.unlock();
        finish_pending(p, LBM_ERR_BUSY, t_tick);
      }
      continue;
    }
    if (changed) {
      std::vector<Member*> ms;
      for (Slot& s : slots) ms.push_back(s.m);
      lbm_status s = engine_set_members(E, ms);
      if (s != LBM_OK) {
        fail_all(s);
        return;
      }
      changed = false;
    }
    const int n = (int)slots.size();
    std::vector<int> which;
    std::vector<int32_t> n_swap;
    for (int i = 0; i < n; ++i)
      if (slots[i].exchange_next) {
        which.push_back(i);
        n_swap.push_back(slots[i].q.r.n_swap);
      }
    std::vector<int64_t> before(n);
    for (int i = 0; i < n; ++i) before[i] = slots[i].m->fluid_cells;
    lbm_status s = LBM_OK;
    if (!which.empty()) s = enqueue_exchange(E, which, n_swap.data());
    int64_t S = cfg.max_tick_steps;
    for (const Slot& x : slots) S = std::min(S, x.steps_left);
    if (s == LBM_OK) s = enqueue_steps_and_reduce(E, S, false);
    if (s == LBM_OK && cudaStreamSynchronize(E->stream) != cudaSuccess)
      s = fail(LBM_ERR_CUDA, "server tick");
    if (s != LBM_OK) {
      fail_all(s == LBM_ERR_OOM ? LBM_ERR_OOM : LBM_ERR_CUDA);
      return;
    }
    std::vector<int32_t> status(n, LBM_OK);
    for (size_t k = 0; k < which.size(); ++k) {
      Slot& x = slots[which[k]];
      x.exchange_next = false;
      x.n_swapped += E->h_info[8 * k];
      if (E->h_info[8 * k + 3] != 0) status[which[k]] = LBM_ERR_DIVERGED;
    }
    if (!which.empty())
      for (int i = 0; i < n; ++i) {
        slots[i].m->fluid_cells = (int64_t)E->h_count[i];
        if (slots[i].m->fluid_cells != before[i]) status[i] = LBM_ERR_CUDA;  // volume not kept
      }
    account_steps(E, S);
    std::vector<bool> retire(n, false);
    for (int i = 0; i < n; ++i) {
      Slot& x = slots[i];
      x.m->steps_done += S;
      x.fluid_updates += S * x.m->fluid_cells;
      x.steps_left -= S;
      if (E->h_result[(size_t)i * kResultDoubles + 7] != 0.0 && status[i] == LBM_OK) status[i] = LBM_ERR_DIVERGED;
      if (status[i] != LBM_OK) {
        fill_result(E, i, &x.last);
        retire[i] = true;
        continue;
      }
      if (x.steps_left > 0) continue;
      fill_result(E, i, &x.last);
      if (!x.first_done) {
        x.dp_first = x.last.dp;
        x.first_done = true;
      }
      if (x.iter < x.q.r.n_iter) {
        ++x.iter;
        x.exchange_next = true;
        x.steps_left = x.q.r.n_steps;
        continue;
      }
      const size_t cells = (size_t)x.m->nx * x.m->ny;
      struct {
        void* dst;
        uint32_t which;
        size_t bytes;
      } outs[4] = {{x.q.r.out_mask, LBM_FIELD_MASK, cells},
                   {x.q.r.out_drho, LBM_FIELD_DRHO, 4 * cells},
                   {x.q.r.out_ux, LBM_FIELD_UX, 4 * cells},
                   {x.q.r.out_uy, LBM_FIELD_UY, 4 * cells}};
      for (auto& o : outs)
        if (o.dst && status[i] == LBM_OK) status[i] = engine_read(E, i, o.which, o.dst, o.bytes);
      retire[i] = true;
    }
    std::vector<Slot> keep;
    for (int i = 0; i < n; ++i) {
      if (retire[i]) {
        finish(slots[i], status[i]);
        delete slots[i].m;
        changed = true;
      } else {
        keep.push_back(std::move(slots[i]));
      }
    }
    slots.swap(keep);
    if (slots.empty()) E->m.clear();  // retired members are gone
    size_t dev_bytes = engine_buffer_bytes(E);
    for (const Slot& x : slots) dev_bytes += x.m->slab_bytes;
    {
      std::lock_guard<std::mutex> lk(mu);
      ++st.ticks;
      st.exchanges += which.empty() ? 0 : 1;
      st.active = (int32_t)slots.size();
      st.peak_active = std::max<int32_t>(st.peak_active, n);
      st.device_bytes = (int64_t)dev_bytes;
      st.peak_device_bytes = std::max<int64_t>(st.peak_device_bytes, st.device_bytes);
      st.busy_s += now() - t_tick;
      st.step_ms = E->step_ms;
      st.fluid_updates = E->fluid_updates;
      cv_done.notify_all();
    }
  }
}

extern "C" {

lbm_status lbm_server_create(const lbm_server_config* cfg, void* cuda_stream, lbm_server* out) {
  if (!out) return fail(LBM_ERR_ARG, "out is NULL");
  *out = nullptr;
  if (!cfg) return fail(LBM_ERR_ARG, "cfg is NULL");
  if (cfg->precision < LBM_F32 || cfg->precision > LBM_F16_SHIFTED) return fail(LBM_ERR_ARG, "precision");
  if (cfg->max_active < 1 || cfg->max_tick_steps < 2 || (cfg->max_tick_steps % 2) != 0 ||
      cfg->hbm_budget_bytes < 0 || cfg->reserved != 0)
    return fail(LBM_ERR_ARG, "max_active >= 1, max_tick_steps even and >= 2, budget >= 0, reserved 0");
  lbm_server s = new lbm_server_s();
  s->cfg = *cfg;
  s->t0 = std::chrono::steady_clock::now();
  cudaError_t e = cudaGetDevice(&s->device);
  size_t free_b = 0, total_b = 0;
  if (e == cudaSuccess) e = cudaMemGetInfo(&free_b, &total_b);
  if (e != cudaSuccess) {
    delete s;
    return fail(LBM_ERR_CUDA, std::string("lbm_server_create: ") + cudaGetErrorString(e));
  }
  s->budget = cfg->hbm_budget_bytes > 0 ? cfg->hbm_budget_bytes : (int64_t)(0.8 * (double)free_b);
  s->st.budget_bytes = s->budget;
  lbm_status st = engine_new(cfg->precision, 0, cuda_stream, true, &s->E);
  if (st != LBM_OK) {
    delete s;
    return st;
  }
  s->E->own_members = false;
  s->th = std::thread([s] { s->loop(); });
  *out = s;
  return LBM_OK;
}

int64_t lbm_server_footprint(const lbm_params* params, int32_t n_iter) {
  if (!params) return -1;
  return footprint_of(*params, n_iter);
}

lbm_status lbm_server_submit(lbm_server s, const lbm_request* r) {
  if (!s || !r) return fail(LBM_ERR_ARG, "server or request is NULL");
  const lbm_params& p = r->params;
  if (p.precision != s->cfg.precision) return fail(LBM_ERR_ARG, "request precision differs from the server's");
  if (p.residual_every != 0) return fail(LBM_ERR_ARG, "served requests take residual_every = 0");
  if (r->n_steps < 2 || (r->n_steps % 2) != 0 || r->n_iter < 0 || r->n_swap < 0)
    return fail(LBM_ERR_ARG, "n_steps even and >= 2, n_iter >= 0, n_swap >= 0");
  lbm_status st = member_check(p, r->cell_types);
  if (st != LBM_OK) return st;
  Pending q;
  q.r = *r;
  q.r.cell_types = nullptr;
  q.footprint = footprint_of(p, r->n_iter);
  if (q.footprint > s->budget) return fail(LBM_ERR_ARG, "request footprint exceeds the server's budget");
  q.cells.assign(r->cell_types, r->cell_types + (size_t)p.nx * p.ny);
  q.t_submit = s->now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    if (s->fatal) return fail(LBM_ERR_CUDA, "the server stopped after a CUDA error");
    s->queue.push_back(std::move(q));
    ++s->st.submitted;
    s->st.queued = (int32_t)s->queue.size();
  }
  s->cv_work.notify_one();
  return LBM_OK;
}

int32_t lbm_server_poll(lbm_server s, lbm_served* out, int32_t max_out, int32_t wait_ms) {
  if (!s || !out || max_out < 1) return 0;
  std::unique_lock<std::mutex> lk(s->mu);
  if (s->done.empty() && wait_ms > 0)
    s->cv_done.wait_for(lk, std::chrono::milliseconds(wait_ms), [&] { return !s->done.empty(); });
  int32_t k = 0;
  while (k < max_out && !s->done.empty()) {
    out[k++] = s->done.front();
    s->done.pop_front();
  }
  return k;
}

lbm_status lbm_server_cancel(lbm_server s, int64_t tag) {
  if (!s) return fail(LBM_ERR_ARG, "server is NULL");
  Pending p;
  bool queued = false;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    for (auto it = s->queue.begin(); it != s->queue.end(); ++it)
      if (it->r.tag == tag) {
        p = std::move(*it);
        s->queue.erase(it);
        queued = true;
        s->st.queued = (int32_t)s->queue.size();
        break;
      }
    if (!queued) {
      if (!s->resident_tags.count(tag)) return fail(LBM_ERR_ARG, "no queued or resident request has this tag");
      s->cancel.insert(tag);
    }
  }
  if (queued) {
    {
      std::lock_guard<std::mutex> lk(s->mu);
      s->resident += p.footprint;  // finish() releases what admission would have charged
      s->resident_cells += cells_of(p);
    }
    s->finish_pending(p, LBM_ERR_CANCELLED, s->now());
  }
  s->cv_work.notify_one();
  return LBM_OK;
}

lbm_status lbm_server_wait_idle(lbm_server s, int32_t timeout_ms) {
  if (!s) return fail(LBM_ERR_ARG, "server is NULL");
  std::unique_lock<std::mutex> lk(s->mu);
  const bool ok = s->cv_done.wait_for(lk, std::chrono::milliseconds(std::max(0, timeout_ms)), [&] {
    return s->fatal || (s->queue.empty() && s->st.submitted == s->st.completed + s->st.failed);
  });
  if (!ok) return fail(LBM_ERR_TIMEOUT, "requests still queued or resident");
  return LBM_OK;
}

lbm_status lbm_server_get_stats(lbm_server s, lbm_server_stats* out) {
  if (!s || !out) return fail(LBM_ERR_ARG, "server or out is NULL");
  std::lock_guard<std::mutex> lk(s->mu);
  *out = s->st;
  return LBM_OK;
}

double lbm_server_now(lbm_server s) { return s ? s->now() : 0.0; }

void lbm_server_destroy(lbm_server s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->th.joinable()) s->th.join();
  for (Slot& x : s->slots) delete x.m;
  s->slots.clear();
  delete s->E;
  delete s;
}

}  // extern "C"
