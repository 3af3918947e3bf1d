// Serving: continuous admission of lambda-sweep and Algorithm 2 requests.
//
// A server keeps forward operators ("problems") resident and runs the
// requests submitted against them on up to max_slots slots.  Each slot is a
// host thread that drives one context (its own CUDA stream, operator copy,
// Galerkin hierarchy and workspace), so the kernels of requests running in
// different slots overlap on the device.  A request is admitted, in arrival
// order among those that fit, as soon as a slot is free and the device
// bytes it needs fit in the HBM budget next to everything resident: an
// idle context of the same problem is reused (operator, hierarchy and the
// last solutions stay resident for warm starts); otherwise a new context is
// created, evicting idle contexts least recently used when room is needed.
// A request that cannot fit even with nothing else resident fails with
// LCMG_ERR_NOMEM.  Every request computes exactly what lcmg_solve /
// lcmg_lcurve_run compute on a fresh context (same kernels, same order of
// every reduction), so its result does not depend on what else runs.
#include <cuda_runtime.h>

#include <algorithm>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <map>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <vector>

#include "lcmg.h"

namespace {

double now_s() {
  using namespace std::chrono;
  return duration<double>(steady_clock::now().time_since_epoch()).count();
}

struct Problem {
  int32_t id = 0;
  int32_t nv = 0, nh = 0, kind = 0;
  int64_t m = 0, n = 0;
  std::vector<int64_t> rp;
  std::vector<int32_t> ci;
  std::vector<float> v32;
  std::vector<double> v64;
  int32_t vdtype = 0;
  int32_t kh = 0, kw = 0;
  std::vector<double> psf;
  int64_t nnz() const { return kind == 0 ? rp[(size_t)m] : 0; }
};

// Device bytes of a context of problem P solving batches of up to B
// columns: operator copies (A and A^T, FP32 values plus FP64 ones when the
// values are FP64), the hierarchy (per-point coefficient rows in FP32 and
// FP64 and the FP64 Galerkin stencils: about 1.6 kB per fine point over all
// levels), the per-column vectors of every level and the coarsest-level
// inverses (coarse side at most 8, 64 points), plus a fixed allowance.
size_t footprint(const Problem& P, int B) {
  const double n = (double)P.n, m = (double)P.m;
  double op = 0;
  if (P.kind == 0) {
    const double nnz = (double)P.nnz();
    op = 2.0 * nnz * (4 + 4 + (P.vdtype ? 8 : 0)) + (m + n + 8) * 8.0;
  } else {
    op = (double)P.kh * P.kw * 12.0;
  }
  const double hier = n * 1600.0;
  const double per_col = n * 160.0 + m * 32.0 + 64.0 * 64.0 * 24.0;
  return (size_t)(op + hier + B * per_col + (64u << 20));
}

struct Request {
  uint64_t ticket = 0;
  int32_t problem = 0;
  std::vector<double> lam, b;
  double tol = 0;
  int32_t max_outer = 0;
  int32_t warm = 0;
  // progress
  int state = 0;  // 0 pending, 1 running, 2 done, 3 cancelled
  int err = LCMG_OK;
  std::string msg;
  double t_submit = 0, t_admit = 0, t_done = 0;
  // results
  std::vector<double> x, rho, eta;
  std::vector<int32_t> iters, status, history;
  int32_t n_outer = 0;
  int64_t n_solves = 0, n_conv = 0;
};

struct Ctx {
  lcmg_ctx* ctx = nullptr;
  int32_t problem = -1;
  int B = 0;           // widest batch its workspace was sized for
  size_t bytes = 0;    // counted against the budget
  bool busy = false;
  uint64_t last_used = 0;
  // warm-start iterates of the last sweep (host copy, per lambda)
  std::vector<double> last_lam, last_x;
};

}  // namespace

struct lcmg_server {
  int device = 0;
  size_t budget = 0;
  int slots = 1;
  lcmg_params prm{};
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  bool stop = false;
  std::map<int32_t, std::shared_ptr<Problem>> problems;
  std::deque<std::shared_ptr<Request>> pending;
  std::map<uint64_t, std::shared_ptr<Request>> all;
  std::vector<std::unique_ptr<Ctx>> ctxs;
  size_t resident = 0;      // bytes of all contexts
  uint64_t next_ticket = 1, clock = 0;
  int32_t next_problem = 0;
  int running = 0, peak_running = 0;
  int64_t admitted = 0, completed = 0, evictions = 0, reuses = 0;
  std::vector<std::thread> workers;
};

namespace {

thread_local std::string s_err;

int fail(int code, const std::string& m) {
  s_err = m;
  return code;
}

int batch_width(const lcmg_params& p, const Request& r) {
  return p.mode == LCMG_MODE_SEQUENTIAL ? 1 : (int)r.lam.size();
}

void destroy_ctx(Ctx& c) {
  if (c.ctx) lcmg_destroy(c.ctx);
  c.ctx = nullptr;
}

// Pick the next request to admit and the context it runs on (server lock
// held).  Returns false when nothing can start now.  `create_bytes` > 0
// means a new context of that many bytes must be created for it.  Idle
// contexts evicted to make room are moved to `evicted` (their bytes already
// released from the account): the caller destroys them after unlocking, so
// submit and wait never stall on a context's teardown.
bool admit_one(lcmg_server& S, std::shared_ptr<Request>& out, Ctx*& ctx_out, size_t& create_bytes,
               std::vector<std::unique_ptr<Ctx>>& evicted) {
  for (auto it = S.pending.begin(); it != S.pending.end(); ++it) {
    Request& r = **it;
    const Problem& P = *S.problems.at(r.problem);
    const int B = batch_width(S.prm, r);
    // an idle context of the same problem, widest first
    Ctx* best = nullptr;
    for (auto& c : S.ctxs)
      if (!c->busy && c->problem == r.problem && (!best || c->B > best->B)) best = c.get();
    if (best) {
      size_t grow = 0;
      if (B > best->B) grow = footprint(P, B) - footprint(P, best->B);
      if (S.resident + grow <= S.budget) {
        best->bytes += grow;
        S.resident += grow;
        best->B = std::max(best->B, B);
        out = *it;
        S.pending.erase(it);
        ctx_out = best;
        create_bytes = 0;
        ++S.reuses;
        return true;
      }
    }
    const size_t need = footprint(P, B);
    if (need > S.budget) {
      // can never fit: fail it now
      r.state = 2;
      r.err = LCMG_ERR_NOMEM;
      r.msg = "request needs about " + std::to_string(need) + " device bytes, over the server budget";
      r.t_done = now_s();
      S.pending.erase(it);
      S.cv_done.notify_all();
      return admit_one(S, out, ctx_out, create_bytes, evicted);
    }
    // evict idle contexts, least recently used first, until it fits; only
    // when evicting every idle one would make it fit (busy contexts keep
    // their bytes), so hierarchies and warm starts are not thrown away for
    // a request that must wait anyway
    size_t idle = 0;
    for (auto& c : S.ctxs)
      if (!c->busy) idle += c->bytes;
    while (S.resident + need > S.budget && S.resident - idle + need <= S.budget) {
      Ctx* lru = nullptr;
      for (auto& c : S.ctxs)
        if (!c->busy && (!lru || c->last_used < lru->last_used)) lru = c.get();
      if (!lru) break;
      S.resident -= lru->bytes;
      idle -= lru->bytes;
      ++S.evictions;
      auto pos = std::find_if(S.ctxs.begin(), S.ctxs.end(), [&](const std::unique_ptr<Ctx>& c) { return c.get() == lru; });
      evicted.push_back(std::move(*pos));
      S.ctxs.erase(pos);
    }
    if (S.resident + need <= S.budget) {
      auto c = std::make_unique<Ctx>();
      c->problem = r.problem;
      c->B = B;
      c->bytes = need;
      c->busy = true;
      S.resident += need;
      ctx_out = c.get();
      S.ctxs.push_back(std::move(c));
      out = *it;
      S.pending.erase(it);
      create_bytes = need;
      return true;
    }
    // does not fit while others run: later requests may still fit
  }
  return false;
}

int make_ctx(lcmg_server& S, const Problem& P, lcmg_ctx** out) {
  lcmg_ctx* c = nullptr;
  int st = lcmg_create(&c, S.device, nullptr, &S.prm);
  if (st != LCMG_OK) return st;
  st = lcmg_set_grid(c, P.nv, P.nh);
  if (st == LCMG_OK) {
    if (P.kind == 0)
      st = lcmg_set_forward_csr(c, P.m, P.n, P.rp.data(), P.ci.data(),
                                P.vdtype ? (const void*)P.v64.data() : (const void*)P.v32.data(), P.vdtype);
    else
      st = lcmg_set_forward_stencil(c, P.kh, P.kw, P.psf.data());
  }
  if (st != LCMG_OK) {
    lcmg_destroy(c);
    return st;
  }
  *out = c;
  return LCMG_OK;
}

// Run one request on its context (no server lock held).
void execute(lcmg_server& S, Request& r, Ctx& C, const Problem& P) {
  lcmg_params p = S.prm;
  if (r.tol > 0) p.tol = r.tol;
  int st = lcmg_set_params(C.ctx, &p);
  // every request starts from D = I
  if (st == LCMG_OK) {
    std::vector<double> ones((size_t)(P.nh * (P.nv - 1) + (P.nh - 1) * P.nv), 1.0);
    st = lcmg_set_weights(C.ctx, ones.data(), (int64_t)ones.size());
  }
  const int nl = (int)r.lam.size();
  if (st == LCMG_OK && r.max_outer == 0) {
    r.x.assign((size_t)P.n * nl, 0.0);
    r.rho.assign(nl, 0.0);
    r.eta.assign(nl, 0.0);
    r.iters.assign(nl, 0);
    r.status.assign(nl, 0);
    const bool warm = r.warm && C.last_lam == r.lam && C.last_x.size() == r.x.size();
    // a warm request starts every lambda from its own resident solution (the
    // chain would start only the largest one there)
    const bool rebatch = warm && S.prm.mode == LCMG_MODE_SEQUENTIAL;
    if (rebatch) {
      lcmg_params p = S.prm;
      p.mode = LCMG_MODE_BATCHED;
      lcmg_set_params(C.ctx, &p);
    }
    st = lcmg_solve(C.ctx, nl, r.lam.data(), 1, r.b.data(), warm ? C.last_x.data() : nullptr, r.x.data(),
                    r.rho.data(), r.eta.data(), r.iters.data(), r.status.data());
    if (rebatch) lcmg_set_params(C.ctx, &S.prm);
    if (st == LCMG_OK) {
      C.last_lam = r.lam;
      C.last_x = r.x;
      r.n_solves = nl;
      for (int j = 0; j < nl; ++j) r.n_conv += r.status[j] == LCMG_CONVERGED;
    }
  } else if (st == LCMG_OK) {
    r.x.assign((size_t)P.n, 0.0);
    r.history.assign(r.max_outer, 0);
    st = lcmg_lcurve_run(C.ctx, nl, r.lam.data(), r.b.data(), r.max_outer, r.x.data(), r.history.data(),
                         &r.n_outer, &r.n_solves, &r.n_conv);
  }
  if (st != LCMG_OK) {
    r.err = st;
    r.msg = lcmg_last_error();
  }
}

void worker(lcmg_server* Sp) {
  lcmg_server& S = *Sp;
  if (cudaSetDevice(S.device) != cudaSuccess) return;
  std::unique_lock<std::mutex> lk(S.mu);
  for (;;) {
    std::shared_ptr<Request> r;
    Ctx* C = nullptr;
    size_t create = 0;
    std::vector<std::unique_ptr<Ctx>> evicted;
    S.cv_work.wait(lk, [&] { return S.stop || admit_one(S, r, C, create, evicted); });
    if (!r) {
      lk.unlock();
      for (auto& e : evicted) destroy_ctx(*e);
      lk.lock();
      if (S.stop) return;
      continue;
    }
    r->state = 1;
    r->t_admit = now_s();
    C->busy = true;
    ++S.running;
    ++S.admitted;
    S.peak_running = std::max(S.peak_running, S.running);
    std::shared_ptr<Problem> P = S.problems.at(r->problem);
    lk.unlock();
    for (auto& e : evicted) destroy_ctx(*e);  // outside the lock
    evicted.clear();
    bool ok = true;
    if (create) {
      const int st = make_ctx(S, *P, &C->ctx);
      if (st != LCMG_OK) {
        r->err = st;
        r->msg = lcmg_last_error();
        ok = false;
      }
    }
    if (ok) execute(S, *r, *C, *P);
    lk.lock();
    r->t_done = now_s();
    r->state = 2;
    --S.running;
    ++S.completed;
    C->busy = false;
    C->last_used = ++S.clock;
    if (!ok) {  // drop the context that could not be built
      S.resident -= C->bytes;
      destroy_ctx(*C);
      S.ctxs.erase(std::find_if(S.ctxs.begin(), S.ctxs.end(), [&](const std::unique_ptr<Ctx>& c) { return c.get() == C; }));
    }
    S.cv_done.notify_all();
    S.cv_work.notify_all();  // a slot and maybe memory are free
  }
}

int copy_result(const Request& r, lcmg_result* out) {
  out->state = r.err;
  out->n_lambda = (int32_t)r.lam.size();
  out->n_outer = r.n_outer;
  out->n_solves = r.n_solves;
  out->n_converged = r.n_conv;
  out->t_submit = r.t_submit;
  out->t_admit = r.t_admit;
  out->t_done = r.t_done;
  if (out->x && !r.x.empty()) std::memcpy(out->x, r.x.data(), sizeof(double) * r.x.size());
  if (out->rho && !r.rho.empty()) std::memcpy(out->rho, r.rho.data(), sizeof(double) * r.rho.size());
  if (out->eta && !r.eta.empty()) std::memcpy(out->eta, r.eta.data(), sizeof(double) * r.eta.size());
  if (out->iters && !r.iters.empty()) std::memcpy(out->iters, r.iters.data(), sizeof(int32_t) * r.iters.size());
  if (out->status && !r.status.empty()) std::memcpy(out->status, r.status.data(), sizeof(int32_t) * r.status.size());
  if (out->history && !r.history.empty())
    std::memcpy(out->history, r.history.data(), sizeof(int32_t) * r.history.size());
  if (r.err != LCMG_OK) s_err = r.msg;
  return LCMG_OK;
}

}  // namespace

extern "C" {

const char* lcmg_server_last_error(void) { return s_err.c_str(); }

int lcmg_server_create(lcmg_server** out, int device, size_t hbm_budget_bytes, int32_t max_slots,
                       const lcmg_params* p) {
  if (!out || max_slots < 1 || max_slots > 64 || hbm_budget_bytes == 0)
    return fail(LCMG_ERR_INVALID_ARG, "server: bad arguments");
  int ndev = 0;
  if (cudaGetDeviceCount(&ndev) != cudaSuccess || device < 0 || device >= ndev) {
    cudaGetLastError();
    return fail(LCMG_ERR_CUDA, "server: no such CUDA device");
  }
  auto S = new lcmg_server();
  S->device = device;
  S->budget = hbm_budget_bytes;
  S->slots = max_slots;
  if (p)
    S->prm = *p;
  else
    lcmg_default_params(&S->prm);
  for (int i = 0; i < max_slots; ++i) S->workers.emplace_back(worker, S);
  *out = S;
  return LCMG_OK;
}

int lcmg_server_add_problem(lcmg_server* S, const lcmg_problem* pr, int32_t* id) {
  if (!S || !pr || !id) return fail(LCMG_ERR_INVALID_ARG, "server: null argument");
  if (pr->n_v < 2 || pr->n_h < 2) return fail(LCMG_ERR_INVALID_ARG, "server: grid sides must be >= 2");
  auto P = std::make_shared<Problem>();
  P->nv = pr->n_v;
  P->nh = pr->n_h;
  P->n = (int64_t)pr->n_v * pr->n_h;
  P->kind = pr->kind;
  if (pr->kind == 0) {
    if (pr->m < 1 || !pr->row_ptr || !pr->col || !pr->val || (pr->val_dtype != 0 && pr->val_dtype != 1))
      return fail(LCMG_ERR_INVALID_ARG, "server: bad CSR problem");
    P->m = pr->m;
    P->rp.assign(pr->row_ptr, pr->row_ptr + pr->m + 1);
    const int64_t nnz = P->rp.back();
    if (nnz < 0) return fail(LCMG_ERR_INVALID_ARG, "server: bad row pointers");
    P->ci.assign(pr->col, pr->col + nnz);
    P->vdtype = pr->val_dtype;
    if (pr->val_dtype == 0) {
      const float* v = static_cast<const float*>(pr->val);
      P->v32.assign(v, v + nnz);
    } else {
      const double* v = static_cast<const double*>(pr->val);
      P->v64.assign(v, v + nnz);
    }
  } else if (pr->kind == 1) {
    if (pr->kh < 1 || pr->kw < 1 || !pr->psf) return fail(LCMG_ERR_INVALID_ARG, "server: bad PSF problem");
    P->m = P->n;
    P->kh = pr->kh;
    P->kw = pr->kw;
    P->psf.assign(pr->psf, pr->psf + (size_t)pr->kh * pr->kw);
  } else {
    return fail(LCMG_ERR_INVALID_ARG, "server: kind must be 0 (CSR) or 1 (PSF)");
  }
  std::lock_guard<std::mutex> lk(S->mu);
  P->id = S->next_problem++;
  S->problems[P->id] = P;
  *id = P->id;
  return LCMG_OK;
}

int lcmg_server_submit(lcmg_server* S, const lcmg_request* rq, uint64_t* ticket) {
  if (!S || !rq || !ticket) return fail(LCMG_ERR_INVALID_ARG, "server: null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto pit = S->problems.find(rq->problem);
  if (pit == S->problems.end()) return fail(LCMG_ERR_INVALID_ARG, "server: unknown problem id");
  const Problem& P = *pit->second;
  if (rq->n_lambda < 1 || !rq->lambda || !rq->b || rq->max_outer < 0 || rq->tol < 0)
    return fail(LCMG_ERR_INVALID_ARG, "server: bad request");
  if (rq->max_outer > 0 && rq->n_lambda < 3) return fail(LCMG_ERR_INVALID_ARG, "server: Algorithm 2 needs >= 3 lambdas");
  auto r = std::make_shared<Request>();
  r->ticket = S->next_ticket++;
  r->problem = rq->problem;
  r->lam.assign(rq->lambda, rq->lambda + rq->n_lambda);
  for (size_t i = 0; i < r->lam.size(); ++i)
    if (!(r->lam[i] > 0) || (i > 0 && !(r->lam[i] > r->lam[i - 1])))
      return fail(LCMG_ERR_INVALID_ARG, "server: lambdas must be positive and increasing");
  r->b.assign(rq->b, rq->b + P.m);
  r->tol = rq->tol;
  r->max_outer = rq->max_outer;
  r->warm = rq->warm;
  r->t_submit = now_s();
  S->pending.push_back(r);
  S->all[r->ticket] = r;
  *ticket = r->ticket;
  S->cv_work.notify_all();
  return LCMG_OK;
}

int lcmg_server_poll(lcmg_server* S, uint64_t ticket, lcmg_result* out) {
  if (!S || !out) return fail(LCMG_ERR_INVALID_ARG, "server: null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return fail(LCMG_ERR_INVALID_ARG, "server: unknown ticket");
  const Request& r = *it->second;
  if (r.state == 3) {
    S->all.erase(it);
    return LCMG_ERR_CANCELLED;
  }
  if (r.state != 2) return LCMG_ERR_NOT_READY;
  copy_result(r, out);
  S->all.erase(it);
  return LCMG_OK;
}

int lcmg_server_wait(lcmg_server* S, uint64_t ticket, double timeout_s, lcmg_result* out) {
  if (!S || !out) return fail(LCMG_ERR_INVALID_ARG, "server: null argument");
  std::unique_lock<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return fail(LCMG_ERR_INVALID_ARG, "server: unknown ticket");
  std::shared_ptr<Request> r = it->second;
  const auto pred = [&] { return r->state >= 2; };
  if (timeout_s > 0) {
    if (!S->cv_done.wait_for(lk, std::chrono::duration<double>(timeout_s), pred)) return LCMG_ERR_NOT_READY;
  } else {
    S->cv_done.wait(lk, pred);
  }
  S->all.erase(ticket);
  if (r->state == 3) return LCMG_ERR_CANCELLED;
  copy_result(*r, out);
  return LCMG_OK;
}

int lcmg_server_cancel(lcmg_server* S, uint64_t ticket) {
  if (!S) return fail(LCMG_ERR_INVALID_ARG, "server: null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->all.find(ticket);
  if (it == S->all.end()) return fail(LCMG_ERR_INVALID_ARG, "server: unknown ticket");
  Request& r = *it->second;
  if (r.state != 0) return fail(LCMG_ERR_STATE, "server: only pending requests can be cancelled");
  S->pending.erase(std::find(S->pending.begin(), S->pending.end(), it->second));
  r.state = 3;
  r.t_done = now_s();
  S->cv_done.notify_all();
  return LCMG_OK;
}

int lcmg_server_get_stats(lcmg_server* S, lcmg_server_stats* out) {
  if (!S || !out) return fail(LCMG_ERR_INVALID_ARG, "server: null argument");
  std::lock_guard<std::mutex> lk(S->mu);
  out->resident_bytes = S->resident;
  out->contexts = (int32_t)S->ctxs.size();
  out->pending = (int32_t)S->pending.size();
  out->running = S->running;
  out->peak_running = S->peak_running;
  out->admitted = S->admitted;
  out->completed = S->completed;
  out->evictions = S->evictions;
  out->reuses = S->reuses;
  return LCMG_OK;
}

int lcmg_server_footprint(lcmg_server* S, int32_t problem, int32_t n_cols, size_t* bytes) {
  if (!S || !bytes || n_cols < 1) return fail(LCMG_ERR_INVALID_ARG, "server: bad arguments");
  std::lock_guard<std::mutex> lk(S->mu);
  auto it = S->problems.find(problem);
  if (it == S->problems.end()) return fail(LCMG_ERR_INVALID_ARG, "server: unknown problem id");
  *bytes = footprint(*it->second, n_cols);
  return LCMG_OK;
}

int lcmg_server_destroy(lcmg_server* S) {
  if (!S) return LCMG_OK;
  {
    std::lock_guard<std::mutex> lk(S->mu);
    S->stop = true;
    for (auto& r : S->pending) {
      r->state = 3;
      r->t_done = now_s();
    }
    S->pending.clear();
  }
  S->cv_work.notify_all();
  S->cv_done.notify_all();
  for (auto& t : S->workers) t.join();
  for (auto& c : S->ctxs) destroy_ctx(*c);
  delete S;
  return LCMG_OK;
}

}  // extern "C"
