// Multi-instance engine: many independent sampling instances (different U, L, N,
// sample counts) advanced together by grouped launches.
//
//   ffs_sample_batched  every instance starts at step 0; the whole schedule (one grouped
//                       init, then per step a grouped residual, a grouped state step and,
//                       at panel ends, a grouped panel update) is captured once into a
//                       CUDA graph and launched as one graph.
//   ffs_server_*        continuous batching: a host thread admits queued requests as HBM
//                       budget and slots free up; each engine iteration advances every
//                       active request by one step (requests sit at different steps), so
//                       new requests overlap on the device with older ones.
//
// Each sample's arithmetic is the same per-sample code as ffs_sample_ex, keyed by its own
// (seed, sample index), so a request's result is the same alone and in any mix.
#include <algorithm>
#include <atomic>
#include <chrono>
#include <condition_variable>
#include <cstring>
#include <deque>
#include <mutex>
#include <thread>
#include <unordered_map>
#include <vector>

#include "ffs_group.cuh"
#include "ffs_residual_tc.cuh"

namespace fermi {

namespace {

constexpr int kPanel = 32;

// Group descriptor of handle c sampling B samples into x (n_steps steps).
void fill_inst(GroupInst& g, ffs_ctx* c, int64_t B, uint64_t seed, uint64_t first, int32_t* x, int64_t n_steps) {
  memset((void*)&g, 0, sizeof g);
  const int op = ctx_op_mode(c);
  g.tm[0] = c->tmH[0];
  g.tm[1] = c->tmH[1];
  g.tm[2] = c->tmU[0];
  g.tm[3] = c->tmU[1];
  StepArgs& a = g.a;
  a.L = c->L;
  a.N = c->N;
  a.Lr = c->Lr;
  a.Kr = c->Kr;
  a.Kp = c->Kp;
  a.ldP = c->ldP;
  a.ldMask = c->ldMask;
  a.bw = B;
  a.n_steps = n_steps;
  a.seed = seed;
  a.first = first;
  a.cplx = c->cplx;
  a.U64 = c->U64;
  a.Ust = c->Ust ? c->Ust : c->U64;
  a.m = c->m;
  a.mask = c->mask;
  a.H = c->H;
  a.hplane = c->ws_B * c->Kp;
  a.P = c->P;
  a.W = c->W;
  a.logp = c->logp;
  a.x = x;
  a.force_x = nullptr;
  a.probs = nullptr;
  a.status = c->status;
  a.ldx = n_steps;
  a.sel_p = nullptr;
  a.nlen = nullptr;
  BlockedArgs& t = g.t;
  t.Nc = n_steps;
  t.W = c->W;
  t.W0P = c->W0P;
  t.Sinv = c->Sinv;
  TcArgs& p = g.tc;
  p.bw = B;
  p.L = c->L;
  p.ldP = c->ldP;
  p.ldMask = c->ldMask;
  p.nK = (int)(c->Kp / residual_k_block(op));
  p.cplx = c->cplx ? 1 : 0;
  p.P = c->P;
  p.mask = c->mask;
  p.status = c->status;
  p.spin = TcArgs{}.spin;  // the record was zeroed above: restore the wait limit
  p.fault = 0;
  g.bn = c->res_bn ? c->res_bn : 256;
  g.n_jtiles = c->Lrp / g.bn;
  g.n_btiles = (B + 127) / 128;
}

// Pick (autotune on first use) the residual column tile of handle c for B samples and
// encode its tensor maps; then fill its group descriptor.
cudaError_t tune_and_fill(GroupInst& g, ffs_ctx* c, int64_t B, uint64_t seed, int32_t* x, int64_t n_steps,
                          cudaStream_t st) {
  const int op = ctx_op_mode(c);
  cudaError_t e = prepare_residual_tc(c, op);
  if (e != cudaSuccess) return e;
  fill_inst(g, c, B, seed, 0, x, n_steps);
  const int bn = residual_tile_for(c, g.a, op, st);
  e = prepare_residual_tc_bn(c, op, bn);
  if (e != cudaSuccess) return e;
  fill_inst(g, c, B, seed, 0, x, n_steps);
  return cudaSuccess;
}

enum LaunchKind { kInit = 0, kResidual = 1, kStep = 2, kPanelS = 3, kPanelUpd = 4 };

struct Launch {
  int kind;
  int64_t off;    // first entry in the entry buffer
  int n;          // entries
  int64_t total;  // work items
  int bn;         // residual column tile of the instances in this launch
};

// Builder of one launch's entry list.
struct LaunchBuilder {
  std::vector<GroupEntry>& ents;
  std::vector<Launch>& launches;
  int kind;
  int64_t off, total = 0;
  int bn = 0;
  LaunchBuilder(std::vector<GroupEntry>& e, std::vector<Launch>& l, int k, int tile = 0)
      : ents(e), launches(l), kind(k), off((int64_t)e.size()), bn(tile) {}
  void add(int inst, int64_t k, int64_t items) {
    if (items <= 0) return;
    ents.push_back(GroupEntry{total, inst, (int32_t)k});
    total += items;
  }
  void done() {
    const int n = (int)((int64_t)ents.size() - off);
    if (n > 0) launches.push_back(Launch{kind, off, n, total, bn});
  }
};

bool panel_end(int64_t k, int64_t Nc) {
  const int64_t k1 = std::min((k / kPanel) * kPanel + kPanel, Nc);
  return k + 1 == k1 && k1 < Nc;  // last step of a panel that has trailing columns
}
int64_t panel_items(int64_t B, int64_t k, int64_t Nc) {
  if (!panel_end(k, Nc)) return 0;
  const int64_t k1 = k + 1;
  return B * ((Nc - k1 + 31) / 32);
}
int64_t panel_s_items(int64_t B, int64_t k, int64_t Nc) { return panel_end(k, Nc) ? B : 0; }
int64_t step_items(int64_t B) {
  const int64_t w = blocked_step_samples_per_cta();
  return (B + w - 1) / w;
}

cudaError_t issue(const Launch& L, const GroupInst* d_inst, const GroupEntry* d_ent, bool cplx, int state, int op,
                  int64_t maxNc, cudaStream_t s) {
  const GroupEntry* e = d_ent + L.off;
  switch (L.kind) {
    case kInit: return launch_group_init(d_inst, e, L.n, L.total, op, s);
    case kResidual: return launch_group_residual(d_inst, e, L.n, L.total, op, L.bn, s);
    case kStep: return launch_group_step(d_inst, e, L.n, L.total, cplx, state, op, maxNc, s);
    case kPanelS: return launch_group_panel_s(d_inst, e, L.n, L.total, cplx, state, s);
    case kPanelUpd: return launch_group_panel(d_inst, e, L.n, L.total, cplx, state, op, s);
  }
  return cudaErrorInvalidValue;
}

}  // namespace
}  // namespace fermi

using namespace fermi;

extern "C" int ffs_sample_batched(ffs_handle* hs, const int64_t* Bs, const uint64_t* seeds, int32_t** outs, int n,
                                  void* cuda_stream) {
  if (!hs || !Bs || !seeds || !outs || n < 1) {
    set_null_handle_error("ffs_sample_batched: need n >= 1 and non-NULL arrays");
    return FFS_E_ARG;
  }
  for (int i = 0; i < n; ++i)
    if (!hs[i]) {
      set_null_handle_error("ffs_sample_batched: NULL handle");
      return FFS_E_ARG;
    }
  ffs_ctx* c0 = hs[0];
  const int op = ctx_op_mode(c0), state = ctx_state_kind(c0);
  const bool cplx = c0->cplx;
  for (int i = 0; i < n; ++i) {
    ffs_ctx* c = hs[i];
    if (!ctx_blocked(c) || ctx_op_mode(c) != op || ctx_state_kind(c) != state || c->cplx != cplx ||
        (c->flags & FFS_FORM_MASK) != FFS_FORM_BATCHED)
      return ctx_fail(c0, FFS_E_ARG,
                      "ffs_sample_batched: all handles must use the same batched tensor-core form, state "
                      "precision and real/complex type");
    if (Bs[i] < 0) return ctx_fail(c0, FFS_E_ARG, "ffs_sample_batched: negative sample count");
    if (Bs[i] > 0 && !ptr_is_device(outs[i]))
      return ctx_fail(c0, FFS_E_ARG, "ffs_sample_batched: outputs must be device memory");
    for (int j = 0; j < i; ++j)
      if (hs[j] == c && Bs[i] > 0 && Bs[j] > 0)
        return ctx_fail(c0, FFS_E_ARG, "ffs_sample_batched: a handle appears twice");
  }
  cudaStream_t st = (cudaStream_t)cuda_stream;

  // Instance table (active instances only) and the static schedule.
  std::vector<GroupInst> inst;
  std::vector<int64_t> Ns, Bv;
  int64_t maxN = 0;
  for (int i = 0; i < n; ++i) {
    if (Bs[i] == 0) continue;
    ffs_ctx* c = hs[i];
    int r = ctx_ensure_workspace(c, Bs[i]);
    if (r != FFS_OK) return r;
    GroupInst g;
    cudaError_t e = tune_and_fill(g, c, Bs[i], seeds[i], outs[i], c->N, st);
    if (e != cudaSuccess) return ctx_fail(c0, FFS_E_CUDA, std::string("ffs_sample_batched: ") + cudaGetErrorString(e));
    inst.push_back(g);
    Ns.push_back(c->N);
    Bv.push_back(Bs[i]);
    maxN = std::max<int64_t>(maxN, c->N);
  }
  if (inst.empty()) return FFS_OK;
  const int ni = (int)inst.size();
  std::vector<GroupEntry> ents;
  std::vector<Launch> launches;
  {
    LaunchBuilder lb(ents, launches, kInit);
    for (int i = 0; i < ni; ++i) lb.add(i, 0, (Bv[i] + 127) / 128);
    lb.done();
  }
  for (int64_t k = 0; k < maxN; ++k) {
    for (int tile : {256, 128}) {
      LaunchBuilder res(ents, launches, kResidual, tile);
      for (int i = 0; i < ni; ++i)
        if (k < Ns[i] && inst[i].bn == tile) res.add(i, k, inst[i].n_btiles * inst[i].n_jtiles);
      res.done();
    }
    LaunchBuilder stp(ents, launches, kStep);
    for (int i = 0; i < ni; ++i)
      if (k < Ns[i]) stp.add(i, k, step_items(Bv[i]));
    stp.done();
    LaunchBuilder pas(ents, launches, kPanelS);
    for (int i = 0; i < ni; ++i)
      if (k < Ns[i]) pas.add(i, k, panel_s_items(Bv[i], k, Ns[i]));
    pas.done();
    LaunchBuilder pan(ents, launches, kPanelUpd);
    for (int i = 0; i < ni; ++i)
      if (k < Ns[i]) pan.add(i, k, panel_items(Bv[i], k, Ns[i]));
    pan.done();
  }

  GroupInst* d_inst = nullptr;
  GroupEntry* d_ent = nullptr;
  cudaError_t e = cudaMalloc((void**)&d_inst, sizeof(GroupInst) * ni);
  if (e == cudaSuccess) e = cudaMalloc((void**)&d_ent, sizeof(GroupEntry) * ents.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_inst, inst.data(), sizeof(GroupInst) * ni, cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(d_ent, ents.data(), sizeof(GroupEntry) * ents.size(), cudaMemcpyHostToDevice, st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  // Capture the schedule and launch it as one graph.
  cudaStream_t cs = nullptr;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t exec = nullptr;
  if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking);
  if (e == cudaSuccess) e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
  if (e == cudaSuccess) {
    cudaError_t le = cudaSuccess;
    for (const Launch& L : launches) {
      le = issue(L, d_inst, d_ent, cplx, state, op, maxN, cs);
      if (le != cudaSuccess) break;
    }
    e = cudaStreamEndCapture(cs, &graph);
    if (le != cudaSuccess) e = le;
  }
  if (e == cudaSuccess) e = cudaGraphInstantiate(&exec, graph, 0);
  if (e == cudaSuccess) e = cudaGraphLaunch(exec, st);
  if (exec) cudaGraphExecDestroy(exec);  // freed once the launched graph completes
  if (graph) cudaGraphDestroy(graph);
  if (cs) cudaStreamDestroy(cs);
  if (d_inst) cudaFreeAsync(d_inst, st);
  if (d_ent) cudaFreeAsync(d_ent, st);
  if (e != cudaSuccess) return ctx_fail(c0, FFS_E_CUDA, std::string("ffs_sample_batched: ") + cudaGetErrorString(e));
  return FFS_OK;
}

// ====================================================================== serving engine
namespace fermi {
namespace {

using Clock = std::chrono::steady_clock;

struct Request {
  uint64_t id = 0;
  std::vector<unsigned char> U;  // host copy of U (row-major L x N, dtype)
  int dtype = 0;
  int64_t L = 0, N = 0, n = 0;
  uint64_t seed = 0;
  int32_t* out = nullptr;
  bool out_dev = false;
  size_t footprint = 0;
  Clock::time_point t_submit, t_done;
  // engine state
  ffs_ctx* h = nullptr;
  int32_t* xdev = nullptr;
  int64_t k = 0;
  bool started = false;
  bool done = false;
  int status = FFS_OK;
  std::string msg;
};

size_t elem_bytes(int dtype) {
  return dtype == FFS_F64 ? 8 : dtype == FFS_C128 ? 16 : dtype == FFS_F32 ? 4 : 8;
}

}  // namespace
}  // namespace fermi

struct ffs_server {
  size_t budget = 0;
  unsigned flags = 0;
  int max_active = 0;
  cudaStream_t stream = nullptr;
  int device = 0;
  std::mutex mu;
  std::condition_variable cv_work, cv_done;
  std::deque<fermi::Request*> pending;
  std::vector<fermi::Request*> active;
  std::unordered_map<uint64_t, fermi::Request*> all;
  uint64_t next_id = 1;
  size_t used = 0;
  bool stop = false;
  std::thread worker;
  // device tables of the current iteration
  fermi::GroupInst* d_inst = nullptr;
  size_t d_inst_cap = 0;
  fermi::GroupEntry* d_ent = nullptr;
  size_t d_ent_cap = 0;
  std::atomic<int64_t> n_active{0};
  std::atomic<uint64_t> iterations{0};
  std::atomic<int64_t> peak_active{0};  // most requests advanced by one engine iteration
};

namespace fermi {
namespace {

// Bytes a request holds on the device while active.
size_t request_footprint(const Request& r, unsigned flags) {
  ffs_ctx probe;
  probe.L = r.L;
  probe.N = r.N;
  probe.cplx = (r.dtype == FFS_C128 || r.dtype == FFS_C64);
  probe.flags = flags;
  probe.Lr = probe.cplx ? 2 * r.L : r.L;
  probe.Kr = probe.cplx ? 2 * r.N : r.N;
  probe.Kp = (probe.Kr + 63) / 64 * 64;
  probe.Lrp = (probe.Lr + 255) / 256 * 256;
  probe.ldP = (r.L + 3) / 4 * 4;
  probe.ldMask = (r.L + 31) / 32;
  size_t fixed = (size_t)r.L * r.N * (probe.cplx ? 16 : 8) +
                 (size_t)probe.Lrp * probe.Kp * ctx_op_elem_bytes(ctx_op_mode(&probe));
  if (ctx_state_kind(&probe) != kStateFP64)  // copy of U in the state type
    fixed += (size_t)r.L * r.N * blocked_elem_bytes(probe.cplx, ctx_state_kind(&probe));
  return fixed + (size_t)r.n * (ctx_per_sample_bytes(&probe) + (size_t)r.N * 4) + ((size_t)1 << 20);
}

void finish(ffs_server* s, Request* r, int status, const std::string& msg) {
  if (r->h) ffs_destroy(r->h);
  r->h = nullptr;
  if (r->xdev) cudaFree(r->xdev);
  r->xdev = nullptr;
  r->status = status;
  r->msg = msg;
  r->t_done = Clock::now();
  std::lock_guard<std::mutex> lk(s->mu);
  s->used -= r->footprint;
  r->done = true;
  s->cv_done.notify_all();
}

// Set up a newly admitted request on the device.
bool admit(ffs_server* s, Request* r) {
  int rc = ffs_create_ex(r->U.data(), r->dtype, r->L, r->N, r->N, s->flags, s->stream, &r->h);
  if (rc != FFS_OK) {
    finish(s, r, rc, ffs_last_error(nullptr));
    return false;
  }
  rc = ctx_ensure_workspace(r->h, r->n);
  cudaError_t e = cudaSuccess;
  if (rc == FFS_OK) e = cudaMalloc((void**)&r->xdev, (size_t)r->n * r->N * 4);
  if (rc == FFS_OK && e == cudaSuccess) {
    GroupInst g;
    e = tune_and_fill(g, r->h, r->n, r->seed, r->xdev, r->N, s->stream);
  }
  if (rc != FFS_OK || e != cudaSuccess) {
    finish(s, r, rc != FFS_OK ? rc : FFS_E_NOMEM, "ffs_submit: could not set up the request on the device");
    return false;
  }
  r->U.clear();
  r->U.shrink_to_fit();
  return true;
}

void engine_loop(ffs_server* s) {
  cudaSetDevice(s->device);
  std::vector<GroupInst> inst;
  std::vector<GroupEntry> ents;
  std::vector<Launch> launches;
  while (true) {
    std::vector<Request*> admitted;
    {
      std::unique_lock<std::mutex> lk(s->mu);
      if (s->active.empty() && s->pending.empty())
        s->cv_work.wait_for(lk, std::chrono::milliseconds(50), [&] { return s->stop || !s->pending.empty(); });
      if (s->stop) break;
      // FIFO admission while the budget and the slots allow
      while (!s->pending.empty() && (int)(s->active.size() + admitted.size()) < s->max_active &&
             s->used + s->pending.front()->footprint <= s->budget) {
        Request* r = s->pending.front();
        s->pending.pop_front();
        s->used += r->footprint;
        admitted.push_back(r);
      }
    }
    for (Request* r : admitted)
      if (admit(s, r)) s->active.push_back(r);
    s->n_active.store((int64_t)s->active.size());
    if (s->active.empty()) continue;

    // One iteration: every active request advances by one step, per real/complex group.
    const unsigned fl = s->flags;
    int64_t advanced = 0;
    for (int g = 0; g < 2; ++g) {
      const bool cplx = g == 1;
      inst.clear();
      ents.clear();
      launches.clear();
      std::vector<Request*> members;
      int64_t maxNc = 0;
      for (Request* r : s->active)
        if (r->h->cplx == cplx) {
          GroupInst gi;
          fill_inst(gi, r->h, r->n, r->seed, 0, r->xdev, r->N);
          inst.push_back(gi);
          members.push_back(r);
          maxNc = std::max<int64_t>(maxNc, r->N);
        }
      if (members.empty()) continue;
      const int ni = (int)members.size();
      {
        LaunchBuilder lb(ents, launches, kInit);
        for (int i = 0; i < ni; ++i)
          if (!members[i]->started) lb.add(i, 0, (members[i]->n + 127) / 128);
        lb.done();
      }
      {
        for (int tile : {256, 128}) {
          LaunchBuilder res(ents, launches, kResidual, tile);
          for (int i = 0; i < ni; ++i)
            if (inst[i].bn == tile) res.add(i, members[i]->k, inst[i].n_btiles * inst[i].n_jtiles);
          res.done();
        }
        LaunchBuilder stp(ents, launches, kStep);
        for (int i = 0; i < ni; ++i) stp.add(i, members[i]->k, step_items(members[i]->n));
        stp.done();
        LaunchBuilder pas(ents, launches, kPanelS);
        for (int i = 0; i < ni; ++i) pas.add(i, members[i]->k, panel_s_items(members[i]->n, members[i]->k, members[i]->N));
        pas.done();
        LaunchBuilder pan(ents, launches, kPanelUpd);
        for (int i = 0; i < ni; ++i) pan.add(i, members[i]->k, panel_items(members[i]->n, members[i]->k, members[i]->N));
        pan.done();
      }
      cudaError_t e = cudaSuccess;
      if (s->d_inst_cap < inst.size()) {
        cudaFree(s->d_inst);
        s->d_inst_cap = inst.size() * 2;
        e = cudaMalloc((void**)&s->d_inst, sizeof(GroupInst) * s->d_inst_cap);
      }
      if (e == cudaSuccess && s->d_ent_cap < ents.size()) {
        cudaFree(s->d_ent);
        s->d_ent_cap = ents.size() * 2;
        e = cudaMalloc((void**)&s->d_ent, sizeof(GroupEntry) * s->d_ent_cap);
      }
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_inst, inst.data(), sizeof(GroupInst) * ni, cudaMemcpyHostToDevice, s->stream);
      if (e == cudaSuccess)
        e = cudaMemcpyAsync(s->d_ent, ents.data(), sizeof(GroupEntry) * ents.size(), cudaMemcpyHostToDevice,
                            s->stream);
      const int op = ctx_op_mode(members[0]->h), state = ctx_state_kind(members[0]->h);
      for (const Launch& L : launches)
        if (e == cudaSuccess) e = issue(L, s->d_inst, s->d_ent, cplx, state, op, maxNc, s->stream);
      if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
      if (e != cudaSuccess) {
        // take the group out of the active set first: once finished, a waiter may free them
        s->active.erase(std::remove_if(s->active.begin(), s->active.end(),
                                       [&](Request* r) {
                                         return std::find(members.begin(), members.end(), r) != members.end();
                                       }),
                        s->active.end());
        for (Request* r : members) finish(s, r, FFS_E_CUDA, std::string("engine: ") + cudaGetErrorString(e));
        continue;
      }
      for (Request* r : members) {
        r->started = true;
        r->k += 1;
      }
      advanced += (int64_t)members.size();
    }
    ++s->iterations;
    if (advanced > s->peak_active.load()) s->peak_active.store(advanced);
    (void)fl;
    // Completed requests: leave the active set first (a waiter may free a finished
    // request at once), then check the device status, copy the samples out, release.
    std::vector<Request*> keep, completed;
    for (Request* r : s->active) (r->k < r->N ? keep : completed).push_back(r);
    s->active.swap(keep);
    s->n_active.store((int64_t)s->active.size());
    for (Request* r : completed) {
      int code = FFS_OK;
      cudaError_t e = cudaMemcpy(r->h->status_host, r->h->status, sizeof(int), cudaMemcpyDeviceToHost);
      if (e == cudaSuccess && *r->h->status_host != 0) code = *r->h->status_host;
      if (e == cudaSuccess)
        e = cudaMemcpy(r->out, r->xdev, (size_t)r->n * r->N * 4, r->out_dev ? cudaMemcpyDeviceToDevice
                                                                               : cudaMemcpyDeviceToHost);
      if (e != cudaSuccess) code = FFS_E_CUDA;
      finish(s, r, code, code == FFS_OK ? "" : "request failed on the device");
    }
  }
}

}  // namespace
}  // namespace fermi

extern "C" {

int ffs_server_create(size_t hbm_budget, unsigned flags, int max_active, void* cuda_stream, ffs_server** out) {
  if (!out) {
    set_null_handle_error("ffs_server_create: out is NULL");
    return FFS_E_ARG;
  }
  *out = nullptr;
  if ((flags & FFS_FORM_MASK) != FFS_FORM_BATCHED || (flags & FFS_TAIL_UNBLOCKED) ||
      ((flags & FFS_RES_MASK) == FFS_RES_FP32)) {
    set_null_handle_error("ffs_server_create: the engine runs the batched tensor-core form with the blocked state");
    return FFS_E_ARG;
  }
  ffs_server* s = new ffs_server();
  s->budget = hbm_budget;
  s->flags = flags;
  s->max_active = max_active > 0 ? max_active : 1 << 20;
  s->stream = (cudaStream_t)cuda_stream;
  cudaGetDevice(&s->device);
  if (hbm_budget == 0) {
    size_t fr = 0, tot = 0;
    cudaMemGetInfo(&fr, &tot);
    s->budget = fr / 10 * 8;
  }
  s->worker = std::thread(fermi::engine_loop, s);
  *out = s;
  return FFS_OK;
}

int ffs_submit(ffs_server* s, const void* U, int dtype, int64_t L, int64_t N, int64_t n_samples, uint64_t seed,
               int32_t* out_x, uint64_t* req_id) {
  if (!s || !U || !out_x || !req_id || N < 1 || L < N || n_samples < 1 || dtype < FFS_F64 || dtype > FFS_C64) {
    set_null_handle_error("ffs_submit: invalid arguments");
    return FFS_E_ARG;
  }
  auto* r = new fermi::Request();
  r->dtype = dtype;
  r->L = L;
  r->N = N;
  r->n = n_samples;
  r->seed = seed;
  r->out = out_x;
  r->out_dev = fermi::ptr_is_device(out_x);
  r->U.resize((size_t)L * N * fermi::elem_bytes(dtype));
  if (cudaMemcpy(r->U.data(), U, r->U.size(), cudaMemcpyDefault) != cudaSuccess) {
    delete r;
    set_null_handle_error("ffs_submit: could not read U");
    return FFS_E_ARG;
  }
  r->footprint = fermi::request_footprint(*r, s->flags);
  if (r->footprint > s->budget) {
    delete r;
    set_null_handle_error("ffs_submit: the request needs more device memory than the engine's budget");
    return FFS_E_NOMEM;
  }
  r->t_submit = fermi::Clock::now();
  {
    std::lock_guard<std::mutex> lk(s->mu);
    r->id = s->next_id++;
    s->all[r->id] = r;
    s->pending.push_back(r);
  }
  s->cv_work.notify_one();
  *req_id = r->id;
  return FFS_OK;
}

int ffs_wait(ffs_server* s, uint64_t req_id, int timeout_ms, double* latency_ms) {
  if (!s) {
    set_null_handle_error("ffs_wait: NULL server");
    return FFS_E_ARG;
  }
  std::unique_lock<std::mutex> lk(s->mu);
  auto it = s->all.find(req_id);
  if (it == s->all.end()) {
    set_null_handle_error("ffs_wait: unknown request");
    return FFS_E_ARG;
  }
  fermi::Request* r = it->second;
  auto pred = [&] { return r->done; };
  if (timeout_ms < 0)
    s->cv_done.wait(lk, pred);
  else if (!s->cv_done.wait_for(lk, std::chrono::milliseconds(timeout_ms), pred))
    return FFS_E_TIMEOUT;
  if (latency_ms) latency_ms[0] = std::chrono::duration<double, std::milli>(r->t_done - r->t_submit).count();
  const int status = r->status;
  if (status != FFS_OK) fermi::set_null_handle_error(r->msg);
  s->all.erase(it);
  delete r;
  return status;
}

int ffs_server_stats(ffs_server* s, int64_t* pending, int64_t* active, int64_t* iterations, size_t* bytes_in_use,
                     int64_t* peak_active) {
  if (!s) return FFS_E_ARG;
  std::lock_guard<std::mutex> lk(s->mu);
  if (peak_active) *peak_active = s->peak_active.load();
  if (pending) *pending = (int64_t)s->pending.size();
  if (active) *active = s->n_active.load();
  if (iterations) *iterations = (int64_t)s->iterations.load();
  if (bytes_in_use) *bytes_in_use = s->used;
  return FFS_OK;
}

void ffs_server_destroy(ffs_server* s) {
  if (!s) return;
  {
    std::lock_guard<std::mutex> lk(s->mu);
    s->stop = true;
  }
  s->cv_work.notify_all();
  if (s->worker.joinable()) s->worker.join();
  for (fermi::Request* r : s->active) {
    if (r->h) ffs_destroy(r->h);
    if (r->xdev) cudaFree(r->xdev);
  }
  for (auto& kv : s->all) delete kv.second;
  cudaFree(s->d_inst);
  cudaFree(s->d_ent);
  delete s;
}

}  // extern "C"
