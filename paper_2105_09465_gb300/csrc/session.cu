// Serving engine: a device-resident request loop with continuous batching.
//
// A request is one lens system (image grid, lens, subhalos, inducing grid,
// source weights v and observed fluxes d) plus a number of iterations. Each
// iteration ray-traces the image, reduces the kernel (out = K v, with the
// row moments of the training forward), forms the residual g = out - d, runs
// the full backward pass (dL/dv, dL/dbeta, lens,
// subhalo and hyperparameter gradients of L = 0.5 |out - d|^2) and takes a
// gradient step v <- v - step dL/dv. All of a request's state stays on the
// device from admission to completion.
//
// A worker thread owns the GPU side. Between iterations it admits pending
// requests while slots (max_slots) and the device-memory budget allow, then
// runs ONE iteration for every active request with one batched launch per
// stage (ray-trace, training forward, moments merge, residual, row-gradient
// merge, scalars, d_v sweep, d_v merge, ray-trace VJP, final sums, update):
// requests of different sizes share the launches and their CTAs overlap on
// the device. A request that reaches its iteration count leaves the batch;
// a host callback on the stream timestamps its completion. Every request is
// summed in an order fixed by its own sizes, so its results are bit-identical
// alone or in any mix.
#include <math.h>

#include <chrono>
#include <condition_variable>
#include <deque>
#include <memory>
#include <mutex>
#include <string>
#include <thread>
#include <unordered_map>
#include <vector>

#include "host.cuh"
#include "problems.cuh"

namespace lr {
namespace {

// out[i] = a[i] - alpha * b[i], batched over problems.
__global__ void axpy_batched_kernel(const __grid_constant__ Batch<AxpyP> B) {
  const int k = batch_find(B, blockIdx.x);
  const AxpyP& P = B.p[k];
  const int64_t i = (int64_t)(blockIdx.x - B.start[k]) * blockDim.x + threadIdx.x;
  if (i < P.n) P.out[i] = fmaf(-P.alpha, P.b[i], P.a[i]);
}

lr_status launch_axpy_batched(const AxpyP* p, int count, cudaStream_t s) {
  for (int b0 = 0; b0 < count; b0 += kMaxBatch) {
    Batch<AxpyP> B;
    B.count = count - b0 < kMaxBatch ? count - b0 : kMaxBatch;
    int64_t tot = 0;
    for (int k = 0; k < B.count; ++k) {
      B.p[k] = p[b0 + k];
      B.start[k] = (int32_t)tot;
      tot += (p[b0 + k].n + 255) / 256;
    }
    B.start[B.count] = (int32_t)tot;
    if (tot == 0) continue;
    axpy_batched_kernel<<<(unsigned)tot, 256, 0, s>>>(B);
    LR_CHECK_CUDA(cudaGetLastError());
  }
  return LR_OK;
}

enum class RState { Pending, Active, Done, Failed };

struct Req {
  uint64_t ticket = 0;
  lr_grid grid{}, ygrid{};
  lr_lens lens{};
  int32_t n_sub = 0, profile = 0, iters = 0;
  float ell = 0.f, var = 0.f, step = 0.f;
  std::vector<float> sub, v0, data;
  int64_t n = 0, m = 0;
  // device memory (one allocation) and the offsets of its parts
  size_t bytes = 0;
  size_t o_beta, o_out, o_data, o_g, o_dx, o_v, o_dv, o_sub, o_dlens, o_dsub, o_scal, o_mom, o_train, o_mrows,
      o_dvp, o_vjp;
  char* dmem = nullptr;
  // problem descriptors of the batched stages
  RtP rt;
  BwArgs train;     // training forward: out and the row moments
  MomMergeP tmerge;
  MergeArgs mrows;  // row gradients from the moments
  ScalP scal;
  BwArgs dv;        // d_v sweep
  DvMergeP dvm;
  RowInfoP tinfo, dinfo;  // row-block boxes of the training forward and the d_v sweep
  VjpP vjp;
  VjpFinalP vfin;
  AxpyP resid, upd;
  int iters_done = 0;
  RState state = RState::Pending;
  lr_status status = LR_OK;
  std::string err;
  double t_submit = 0, t_admit = 0, t_done = 0;
  struct lr_session* owner = nullptr;
};

}  // namespace
}  // namespace lr

using namespace lr;

struct lr_session {
  lr_session_cfg cfg{};
  cudaStream_t stream = nullptr, copy_stream = nullptr;
  cudaMemPool_t pool = nullptr;
  cudaEvent_t iter_ev[2] = {nullptr, nullptr};
  std::thread worker;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<Req*> pending;
  std::vector<Req*> active;
  std::unordered_map<uint64_t, std::unique_ptr<Req>> reqs;
  uint64_t next_ticket = 1;
  size_t used = 0;
  bool stop = false;
  bool fault_pending = false;
  uint64_t iterations = 0, launches = 0;
  int64_t peak_pairs = 0;
  std::chrono::steady_clock::time_point t0;
  std::string worker_error;

  double now() const {
    return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
  }
};

namespace {

size_t carve(size_t& off, size_t bytes) {
  const size_t o = off;
  off += align256(bytes);
  return o;
}

// Sizes the request's device state (same plans as the single-problem calls).
lr_status size_request(Req* r) {
  const int64_t n = r->n, m = r->m;
  size_t train_b = 0, mrows_b = 0, dv_b = 0;
  lr_status st = make_train_problem(nullptr, n, &r->grid, nullptr, &r->ygrid, m, nullptr, r->ell, r->var, nullptr,
                                    nullptr, nullptr, nullptr, nullptr, nullptr, &train_b);
  if (st != LR_OK) return st;
  st = make_moment_rows_problem(nullptr, n, true, nullptr, nullptr, r->ell, r->var, nullptr, nullptr, nullptr,
                                nullptr, nullptr, nullptr, &mrows_b);
  if (st != LR_OK) return st;
  st = make_dv_problem(nullptr, n, &r->grid, &r->ygrid, nullptr, r->ell, r->var, nullptr, nullptr, nullptr, nullptr,
                       nullptr, &dv_b);
  if (st != LR_OK) return st;
  size_t off = 0;
  r->o_beta = carve(off, 8 * n);
  r->o_out = carve(off, 4 * n);
  r->o_data = carve(off, 4 * n);
  r->o_g = carve(off, 4 * n);
  r->o_dx = carve(off, 8 * n);
  r->o_v = carve(off, 4 * m);
  r->o_dv = carve(off, 4 * m);
  r->o_sub = carve(off, 20 * (size_t)r->n_sub);
  r->o_dlens = carve(off, 7 * 8);
  r->o_dsub = carve(off, 32 * (size_t)r->n_sub);
  r->o_scal = carve(off, 16);
  r->o_mom = carve(off, 16 * n);
  r->o_train = carve(off, train_b);
  r->o_mrows = carve(off, mrows_b);
  r->o_dvp = carve(off, dv_b);
  r->o_vjp = carve(off, raytrace_vjp_ws(n, r->n_sub));
  r->bytes = off;
  return LR_OK;
}

// Allocates and fills the request's device state and builds its problems.
lr_status init_request(lr_session* S, Req* r) {
  void* p = nullptr;
  LR_CHECK_CUDA(cudaMallocFromPoolAsync(&p, r->bytes, S->pool, S->stream));
  r->dmem = static_cast<char*>(p);
  char* d = r->dmem;
  float2* beta = reinterpret_cast<float2*>(d + r->o_beta);
  float* out = reinterpret_cast<float*>(d + r->o_out);
  float* data = reinterpret_cast<float*>(d + r->o_data);
  float* g = reinterpret_cast<float*>(d + r->o_g);
  float2* dx = reinterpret_cast<float2*>(d + r->o_dx);
  float* v = reinterpret_cast<float*>(d + r->o_v);
  float* dv = reinterpret_cast<float*>(d + r->o_dv);
  float* sub = r->n_sub ? reinterpret_cast<float*>(d + r->o_sub) : nullptr;
  double* dlens = reinterpret_cast<double*>(d + r->o_dlens);
  double* dsub = reinterpret_cast<double*>(d + r->o_dsub);
  double* scal = reinterpret_cast<double*>(d + r->o_scal);
  LR_CHECK_CUDA(cudaMemcpyAsync(v, r->v0.data(), 4 * r->m, cudaMemcpyHostToDevice, S->stream));
  LR_CHECK_CUDA(cudaMemcpyAsync(data, r->data.data(), 4 * r->n, cudaMemcpyHostToDevice, S->stream));
  if (r->n_sub)
    LR_CHECK_CUDA(cudaMemcpyAsync(sub, r->sub.data(), 20 * (size_t)r->n_sub, cudaMemcpyHostToDevice, S->stream));
  lr_status st;
  lr_points P{};
  P.xy = nullptr;
  P.grid = r->grid;
  P.n = r->n;
  P.lens = &r->lens;
  P.sub = sub;
  P.n_sub = r->n_sub;
  P.profile = r->profile;
  if ((st = make_rt_problem(&P, beta, nullptr, &r->rt)) != LR_OK) return st;
  size_t b = 0;
  float* mom = reinterpret_cast<float*>(d + r->o_mom);
  if ((st = make_train_problem(beta, r->n, &r->grid, nullptr, &r->ygrid, r->m, v, r->ell, r->var, out, mom,
                               d + r->o_train, &r->train, &r->tmerge, &r->tinfo, &b)) != LR_OK)
    return st;
  r->resid = AxpyP{out, data, g, r->n, 1.0f};
  if ((st = make_moment_rows_problem(mom, r->n, true, g, v, r->ell, r->var, dx, scal, scal + 1, d + r->o_mrows,
                                     &r->mrows, &r->scal, &b)) != LR_OK)
    return st;
  if ((st = make_dv_problem(beta, r->n, &r->grid, &r->ygrid, g, r->ell, r->var, dv, d + r->o_dvp, &r->dv, &r->dvm,
                            &r->dinfo, &b)) != LR_OK)
    return st;
  if ((st = make_vjp_problem(&P, dx, dlens, dsub, d + r->o_vjp, &r->vjp, &r->vfin)) != LR_OK) return st;
  r->upd = AxpyP{v, dv, v, r->m, r->step};
  return LR_OK;
}

// One batched iteration over `act`.
lr_status run_iteration(lr_session* S, const std::vector<Req*>& act) {
  std::vector<RtP> rt;
  std::vector<RowInfoP> infos;
  std::vector<BwArgs> train, dvs;
  std::vector<MomMergeP> tmerge;
  std::vector<DvMergeP> dvm;
  std::vector<AxpyP> resid, upd;
  std::vector<MergeArgs> mrows;
  std::vector<ScalP> scal;
  std::vector<VjpP> vjp;
  std::vector<VjpFinalP> vfin;
  for (Req* r : act) {
    rt.push_back(r->rt);
    infos.push_back(r->tinfo);
    infos.push_back(r->dinfo);
    train.push_back(r->train);
    tmerge.push_back(r->tmerge);
    resid.push_back(r->resid);
    mrows.push_back(r->mrows);
    scal.push_back(r->scal);
    dvs.push_back(r->dv);
    dvm.push_back(r->dvm);
    vjp.push_back(r->vjp);
    vfin.push_back(r->vfin);
    upd.push_back(r->upd);
  }
  const int n = (int)act.size();
  cudaStream_t s = S->stream;
  lr_status st;
  if ((st = launch_raytrace_batched(rt.data(), n, s)) != LR_OK) return st;
  if ((st = launch_row_info_batched(infos.data(), (int)infos.size(), s)) != LR_OK) return st;
  if ((st = launch_bwd_rows_batched(train.data(), n, s)) != LR_OK) return st;
  if ((st = launch_moments_merge_batched(tmerge.data(), n, s)) != LR_OK) return st;
  if ((st = launch_axpy_batched(resid.data(), n, s)) != LR_OK) return st;
  // d_v (side stream) and the row gradients with the ray-trace VJP are
  // independent branches; the update waits for both
  Fork f{};
  if ((st = fork_begin(s, &f)) != LR_OK) return st;
  st = launch_dv_rows_batched(dvs.data(), n, f.side);
  if (st == LR_OK) st = launch_dv_merge_batched(dvm.data(), n, f.side);
  if (st == LR_OK) st = launch_bwd_merge_batched(mrows.data(), n, s);
  if (st == LR_OK) st = launch_scalar_batched(scal.data(), n, s);
  if (st == LR_OK) st = launch_vjp_batched(vjp.data(), n, s);
  if (st == LR_OK) st = launch_vjp_final_batched(vfin.data(), n, s);
  const lr_status sj = fork_end(s, &f);
  if (st != LR_OK) return st;
  if (sj != LR_OK) return sj;
  if ((st = launch_axpy_batched(upd.data(), n, s)) != LR_OK) return st;
  const int groups = (n + kMaxBatch - 1) / kMaxBatch;
  S->launches += (uint64_t)groups * 11 + (uint64_t)((2 * n + kMaxBatch - 1) / kMaxBatch);
  return LR_OK;
}

void CUDART_CB on_request_done(void* arg) {
  Req* r = static_cast<Req*>(arg);
  lr_session* S = r->owner;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    r->t_done = S->now();
    r->state = RState::Done;
  }
  S->cv_done.notify_all();
}

void fail_request(lr_session* S, Req* r, lr_status st, const std::string& why) {
  // caller holds S->mu
  r->state = RState::Failed;
  r->status = st;
  r->err = why;
  r->t_done = S->now();
  if (r->dmem) {
    cudaFreeAsync(r->dmem, S->stream);
    r->dmem = nullptr;
  }
  S->used -= r->bytes;
}

void worker_main(lr_session* S) {
  cudaSetDevice(S->cfg.device);
  uint64_t k = 0;
  for (;;) {
    std::vector<Req*> admitted;
    std::vector<Req*> act;
    bool inject = false;
    {
      std::unique_lock<std::mutex> lock(S->mu);
      S->cv_work.wait_for(lock, std::chrono::milliseconds(20),
                          [&] { return S->stop || !S->pending.empty() || !S->active.empty(); });
      if (S->stop) break;
      // admission: FIFO while a slot, the memory budget and (when set) the
      // pairs per iteration allow
      int64_t work = 0;
      for (const Req* a : S->active) work += a->n * a->m;
      while (!S->pending.empty() && (int)S->active.size() < S->cfg.max_slots) {
        Req* r = S->pending.front();
        if (S->used + r->bytes > S->cfg.hbm_budget_bytes) break;
        if (S->cfg.fill_pairs > 0 && !S->active.empty() && work + r->n * r->m > S->cfg.fill_pairs) break;
        work += r->n * r->m;
        if (work > S->peak_pairs) S->peak_pairs = work;
        S->pending.pop_front();
        S->used += r->bytes;
        r->state = RState::Active;
        r->t_admit = S->now();
        S->active.push_back(r);
        admitted.push_back(r);
      }
      if (S->active.empty()) continue;
      inject = S->fault_pending;
      S->fault_pending = false;
    }
    for (Req* r : admitted) {
      const lr_status st = init_request(S, r);
      if (st != LR_OK) {
        std::lock_guard<std::mutex> lock(S->mu);
        fail_request(S, r, st, lr_last_error());
      }
    }
    {
      std::lock_guard<std::mutex> lock(S->mu);
      for (Req* r : S->active)
        if (r->state == RState::Active) act.push_back(r);
    }
    // at most two iterations in flight on the stream
    if (k >= 2) cudaEventSynchronize(S->iter_ev[k & 1]);
    lr_status st = inject ? LR_ERR_CUDA : run_iteration(S, act);
    if (inject) set_error("injected fault: the batched iteration was abandoned");
    {
      std::lock_guard<std::mutex> lock(S->mu);
      if (st != LR_OK) {
        const std::string why = lr_last_error();
        for (Req* r : act) fail_request(S, r, st, why);
      } else {
        for (Req* r : act) {
          if (++r->iters_done == r->iters) cudaLaunchHostFunc(S->stream, on_request_done, r);
        }
        ++S->iterations;
      }
      std::vector<Req*> keep;
      for (Req* r : S->active)
        if (r->state == RState::Active && r->iters_done < r->iters) keep.push_back(r);
      S->active.swap(keep);
    }
    cudaEventRecord(S->iter_ev[k & 1], S->stream);
    ++k;
    S->cv_done.notify_all();
  }
}

}  // namespace

extern "C" lr_status solve_session_create(const lr_session_cfg* cfg, lr_session** out) {
  LR_REQUIRE(cfg != nullptr && out != nullptr, "solve_session_create: NULL argument");
  LR_REQUIRE(cfg->max_slots >= 1, "solve_session_create: max_slots = %d must be >= 1", cfg->max_slots);
  LR_REQUIRE(cfg->fill_pairs >= 0, "solve_session_create: fill_pairs < 0");
  auto S = std::make_unique<lr_session>();
  S->cfg = *cfg;
  if (S->cfg.hbm_budget_bytes == 0) S->cfg.hbm_budget_bytes = size_t(120) << 30;
  LR_CHECK_CUDA(cudaSetDevice(cfg->device));
  LR_CHECK_CUDA(cudaStreamCreateWithFlags(&S->stream, cudaStreamNonBlocking));
  LR_CHECK_CUDA(cudaStreamCreateWithFlags(&S->copy_stream, cudaStreamNonBlocking));
  for (auto& e : S->iter_ev) LR_CHECK_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  cudaMemPoolProps props{};
  props.allocType = cudaMemAllocationTypePinned;
  props.location.type = cudaMemLocationTypeDevice;
  props.location.id = cfg->device;
  LR_CHECK_CUDA(cudaMemPoolCreate(&S->pool, &props));
  uint64_t keep = UINT64_MAX;  // keep freed blocks in the pool between requests
  LR_CHECK_CUDA(cudaMemPoolSetAttribute(S->pool, cudaMemPoolAttrReleaseThreshold, &keep));
  S->t0 = std::chrono::steady_clock::now();
  lr_session* raw = S.release();
  raw->worker = std::thread(worker_main, raw);
  *out = raw;
  return LR_OK;
}

extern "C" lr_status solve_session_submit(lr_session* S, const lr_request* q, uint64_t* ticket) {
  LR_REQUIRE(S != nullptr && q != nullptr && ticket != nullptr, "solve_session_submit: NULL argument");
  LR_REQUIRE(q->iters >= 1, "solve_session_submit: iters = %d must be >= 1", q->iters);
  LR_REQUIRE(isfinite(q->lengthscale) && q->lengthscale > 0.f, "solve_session_submit: lengthscale must be > 0");
  LR_REQUIRE(isfinite(q->variance) && isfinite(q->step), "solve_session_submit: variance and step must be finite");
  LR_REQUIRE(q->n_sub >= 0 && (q->n_sub == 0 || q->sub != nullptr), "solve_session_submit: bad subhalo array");
  LR_REQUIRE(q->profile == LR_PROFILE_TNFW || q->profile == LR_PROFILE_POINT_MASS,
             "solve_session_submit: unknown profile %d", q->profile);
  auto r = std::make_unique<Req>();
  r->grid = q->grid;
  r->ygrid = q->ygrid;
  r->lens = q->lens;
  r->n_sub = q->n_sub;
  r->profile = q->profile;
  r->iters = q->iters;
  r->ell = q->lengthscale;
  r->var = q->variance;
  r->step = q->step;
  r->n = grid_count(q->grid);
  r->m = grid_count(q->ygrid);
  lr_points P{};
  P.grid = q->grid;
  P.n = r->n;
  P.lens = &q->lens;
  P.n_sub = 0;
  lr_status st = validate_points(&P, "solve_session_submit(image grid)", true);
  if (st != LR_OK) return st;
  lr_points Y{};
  Y.grid = q->ygrid;
  Y.n = r->m;
  if ((st = validate_points(&Y, "solve_session_submit(inducing grid)", false)) != LR_OK) return st;
  LensConst L;
  if ((st = make_lens_const(&q->lens, &L)) != LR_OK) return st;
  LR_REQUIRE(r->n > 0 && r->m > 0, "solve_session_submit: empty grid");
  LR_REQUIRE(q->v0 != nullptr && q->data != nullptr, "solve_session_submit: v0 and data are required");
  r->v0.assign(q->v0, q->v0 + r->m);
  r->data.assign(q->data, q->data + r->n);
  if (q->n_sub) r->sub.assign(q->sub, q->sub + 5 * (size_t)q->n_sub);
  LR_CHECK_CUDA(cudaSetDevice(S->cfg.device));
  if ((st = size_request(r.get())) != LR_OK) return st;
  if (r->bytes > S->cfg.hbm_budget_bytes) {
    set_error("solve_session_submit: request needs %zu bytes of device memory, the session budget is %zu",
              r->bytes, S->cfg.hbm_budget_bytes);
    return LR_ERR_OUT_OF_MEMORY;
  }
  r->owner = S;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    r->ticket = S->next_ticket++;
    r->t_submit = S->now();
    *ticket = r->ticket;
    S->pending.push_back(r.get());
    S->reqs.emplace(r->ticket, std::move(r));
  }
  S->cv_work.notify_one();
  return LR_OK;
}

extern "C" lr_status solve_session_poll(lr_session* S, uint64_t ticket, lr_result* res, int64_t timeout_us) {
  LR_REQUIRE(S != nullptr && res != nullptr, "solve_session_poll: NULL argument");
  std::unique_lock<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("solve_session_poll: unknown ticket %llu", (unsigned long long)ticket);
    return LR_ERR_NOT_FOUND;
  }
  Req* r = it->second.get();
  auto finished = [&] { return r->state == RState::Done || r->state == RState::Failed; };
  if (!finished()) {
    if (timeout_us <= 0) return LR_PENDING;
    if (!S->cv_done.wait_for(lock, std::chrono::microseconds(timeout_us), finished)) {
      set_error("solve_session_poll: ticket %llu not finished within %lld us", (unsigned long long)ticket,
                (long long)timeout_us);
      return LR_ERR_TIMEOUT;
    }
  }
  res->t_submit_s = r->t_submit;
  res->t_admit_s = r->t_admit;
  res->t_done_s = r->t_done;
  if (r->state == RState::Failed) {
    const lr_status st = r->status;
    set_error("%s", r->err.c_str());
    S->reqs.erase(it);
    return st;
  }
  lock.unlock();
  // results: the request's stream work is complete (its host callback ran)
  std::vector<float> out(r->n);
  char* d = r->dmem;
  cudaStream_t cs = S->copy_stream;
  LR_CHECK_CUDA(cudaMemcpyAsync(out.data(), d + r->o_out, 4 * r->n, cudaMemcpyDeviceToHost, cs));
  if (res->v) LR_CHECK_CUDA(cudaMemcpyAsync(res->v, d + r->o_v, 4 * r->m, cudaMemcpyDeviceToHost, cs));
  if (res->d_lens) LR_CHECK_CUDA(cudaMemcpyAsync(res->d_lens, d + r->o_dlens, 56, cudaMemcpyDeviceToHost, cs));
  if (res->d_sub && r->n_sub)
    LR_CHECK_CUDA(cudaMemcpyAsync(res->d_sub, d + r->o_dsub, 32 * (size_t)r->n_sub, cudaMemcpyDeviceToHost, cs));
  double scal[2];
  LR_CHECK_CUDA(cudaMemcpyAsync(scal, d + r->o_scal, 16, cudaMemcpyDeviceToHost, cs));
  LR_CHECK_CUDA(cudaStreamSynchronize(cs));
  LR_CHECK_CUDA(cudaFreeAsync(r->dmem, cs));
  r->dmem = nullptr;
  double loss = 0.0;
  for (int64_t i = 0; i < r->n; ++i) {
    const double e = (double)out[i] - (double)r->data[i];
    loss += 0.5 * e * e;
  }
  if (res->out) memcpy(res->out, out.data(), 4 * r->n);
  res->d_lengthscale = scal[0];
  res->d_variance = scal[1];
  res->loss = loss;
  lock.lock();
  S->used -= r->bytes;
  S->reqs.erase(ticket);
  lock.unlock();
  S->cv_work.notify_one();
  return LR_OK;
}

extern "C" lr_status solve_session_cancel(lr_session* S, uint64_t ticket) {
  LR_REQUIRE(S != nullptr, "solve_session_cancel: NULL session");
  std::lock_guard<std::mutex> lock(S->mu);
  auto it = S->reqs.find(ticket);
  if (it == S->reqs.end()) {
    set_error("solve_session_cancel: unknown ticket %llu", (unsigned long long)ticket);
    return LR_ERR_NOT_FOUND;
  }
  Req* r = it->second.get();
  if (r->state != RState::Pending) {
    set_error("solve_session_cancel: ticket %llu is already running or finished", (unsigned long long)ticket);
    return LR_ERR_BUSY;
  }
  for (auto p = S->pending.begin(); p != S->pending.end(); ++p)
    if (*p == r) {
      S->pending.erase(p);
      break;
    }
  S->reqs.erase(it);
  return LR_OK;
}

extern "C" lr_status solve_session_inject_fault(lr_session* S) {
  LR_REQUIRE(S != nullptr, "solve_session_inject_fault: NULL session");
  std::lock_guard<std::mutex> lock(S->mu);
  S->fault_pending = true;
  return LR_OK;
}

extern "C" lr_status solve_session_stats(lr_session* S, lr_session_stats* st) {
  LR_REQUIRE(S != nullptr && st != nullptr, "solve_session_stats: NULL argument");
  std::lock_guard<std::mutex> lock(S->mu);
  st->pending = (int64_t)S->pending.size();
  st->active = (int64_t)S->active.size();
  st->held = (int64_t)S->reqs.size() - st->pending - st->active;
  st->used_bytes = S->used;
  st->iterations = S->iterations;
  st->launches = S->launches;
  st->active_pairs = 0;
  for (const Req* r : S->active) st->active_pairs += r->n * r->m;
  st->peak_active_pairs = S->peak_pairs;
  return LR_OK;
}

extern "C" lr_status solve_session_destroy(lr_session* S) {
  if (!S) return LR_OK;
  {
    std::lock_guard<std::mutex> lock(S->mu);
    S->stop = true;
  }
  S->cv_work.notify_all();
  if (S->worker.joinable()) S->worker.join();
  cudaSetDevice(S->cfg.device);
  cudaStreamSynchronize(S->stream);
  for (auto& kv : S->reqs)
    if (kv.second->dmem) cudaFreeAsync(kv.second->dmem, S->stream);
  cudaStreamSynchronize(S->stream);
  cudaStreamSynchronize(S->copy_stream);
  for (auto& e : S->iter_ev) cudaEventDestroy(e);
  cudaStreamDestroy(S->stream);
  cudaStreamDestroy(S->copy_stream);
  cudaMemPoolDestroy(S->pool);
  delete S;
  return LR_OK;
}
