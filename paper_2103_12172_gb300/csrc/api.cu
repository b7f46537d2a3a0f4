// C ABI of the library (declared in include/mdp.h): plan lifetime, batched projection
// columns, the adjoint, full-grid solves, status and host introspection.
#include "mdp_internal.h"
#include "mdp_probe.h"

#include <algorithm>
#include <array>
#include <cstdlib>
#include <cstring>
#include <new>

using namespace mdp;

namespace {

#define CK(x)                                        \
  do {                                               \
    if ((x) != cudaSuccess) return MDP_ERR_CUDA;     \
  } while (0)

long long env_ll(const char *name, long long dflt) {
  const char *v = std::getenv(name);
  if (!v || !*v) return dflt;
  return std::atoll(v);
}

void free_device(mdp_plan *p) {
  if (p->device < 0) return;
  int prev = -1;
  cudaGetDevice(&prev);
  cudaSetDevice(p->device);
  cudaFree(p->d_subs);
  cudaFree(p->d_tables);
  cudaFree(p->d_piv);
  cudaFree(p->d_ws);
  cudaFree(p->d_status);
  cudaFree(p->d_fstatus);
  p->d_fstatus = nullptr;
  p->sub_stage.release();
  p->h_fstatus.release();
  cudaFree(p->alt_subs);
  cudaFree(p->alt_tables);
  cudaFree(p->alt_piv);
  p->alt_subs = nullptr; p->alt_tables = nullptr; p->alt_piv = nullptr;
  p->alt_stage.release();
  for (int s_ = 0; s_ < 2; ++s_) {
    if (p->ready_ev[s_]) cudaEventDestroy(p->ready_ev[s_]);
    if (p->used_ev[s_]) cudaEventDestroy(p->used_ev[s_]);
    p->ready_ev[s_] = p->used_ev[s_] = nullptr;
    p->used_rec[s_] = false;
  }
  for (int k = 0; k < 3; ++k) {
    for (auto x : p->d_items[k]) cudaFree(x);
    for (auto x : p->d_prefix[k]) cudaFree(x);
    for (auto x : p->d_order[k]) cudaFree(x);
    p->d_items[k].clear();
    p->d_prefix[k].clear();
    p->d_order[k].clear();
  }
  p->d_subs = nullptr; p->d_tables = nullptr; p->d_piv = nullptr; p->d_ws = nullptr; p->d_status = nullptr;
  if (prev >= 0) cudaSetDevice(prev);
}

mdp_status upload_subs_tables(mdp_plan *p) {
  std::vector<SubDesc> ds;
  for (auto &hs : p->subs) ds.push_back(hs.d);
  CK(cudaMemcpy(p->d_subs, ds.data(), ds.size() * sizeof(SubDesc), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->d_tables, p->host_tables.data(), p->host_tables.size() * sizeof(double), cudaMemcpyHostToDevice));
  CK(cudaMemcpy(p->d_piv, p->host_piv.data(), p->host_piv.size(), cudaMemcpyHostToDevice));
  return MDP_OK;
}

mdp_status alloc_device(mdp_plan *p) {
  CK(cudaGetDevice(&p->device));
  CK(cudaDeviceGetAttribute(&p->n_sm, cudaDevAttrMultiProcessorCount, p->device));
  CK(set_kernel_attributes());
  auto al = [&](void **ptr, size_t bytes) -> bool { return cudaMalloc(ptr, std::max<size_t>(bytes, 256)) == cudaSuccess; };
  if (!al((void **)&p->d_subs, p->subs.size() * sizeof(SubDesc)) ||
      !al((void **)&p->d_tables, p->host_tables.size() * sizeof(double)) ||
      !al((void **)&p->d_piv, p->host_piv.size()) || !al((void **)&p->d_ws, (size_t)p->ws_doubles * 8) ||
      !al((void **)&p->d_status, sizeof(int)) || !al((void **)&p->d_fstatus, sizeof(int)) ||
      !p->sub_stage.alloc(p->subs.size(), true) || !p->h_fstatus.alloc(1, true))
    return MDP_ERR_NOMEM;
  CK(cudaMemset(p->d_status, 0, sizeof(int)));
  CK(cudaMemset(p->d_fstatus, 0, sizeof(int)));
  for (auto &hs : p->subs) hs.d.dstatus = p->d_status;
#if MDP_CHECKED
  // fault injection (bounds-checked build only): MDP_FAULT_INJECT=factor scales one row of the
  // first subdomain's factored sweep table (row 5 of mode 1, which every projection column goes
  // through: wrong numbers, which the parity check must catch), =desc points the first
  // projection item's mode-space slice past the end of the workspace (the checks must catch it and
  // skip every access through it)
  const char *fault = std::getenv("MDP_FAULT_INJECT");
  if (fault && !std::strcmp(fault, "factor") && !p->subs.empty() && p->subs[0].d.NYf > 6)
    for (int j = 0; j < FSW; ++j) p->host_tables[p->subs[0].d.fs_off + 5 * FSW + j] *= 1.5;
#endif
  mdp_status st = upload_subs_tables(p);
  if (st != MDP_OK) return st;
  for (int sc = 0; sc < 3; ++sc) {
    auto &waves = p->sched[sc];
    auto &ditems = p->d_items[sc];
    auto &dpre = p->d_prefix[sc];
    auto &hpre = p->h_prefix[sc];
    hpre.clear();
    for (auto &w : waves) {
      const int n = (int)w.items.size();
      Item *di = nullptr;
      int *dp = nullptr;
      if (!al((void **)&di, n * sizeof(Item))) return MDP_ERR_NOMEM;
      ditems.push_back(di);
      if (!al((void **)&dp, (size_t)NFAM * (n + 1) * sizeof(int))) return MDP_ERR_NOMEM;
      dpre.push_back(dp);
      std::vector<int> pre((size_t)NFAM * (n + 1), 0);
      for (int f = 0; f < NFAM; ++f)
        for (int i = 0; i < n; ++i)
          pre[(size_t)f * (n + 1) + i + 1] =
              pre[(size_t)f * (n + 1) + i] + blocks_for((Fam)f, p->subs[w.items[i].sub].d, w.items[i].ncols);
#if MDP_CHECKED
      if (fault && !std::strcmp(fault, "desc") && sc == S_PROJ && &w == &waves.front() && n > 0) {
        std::vector<Item> bad(w.items);
        bad[0].y_off = p->ws_doubles;
        CK(cudaMemcpy(di, bad.data(), n * sizeof(Item), cudaMemcpyHostToDevice));
      } else
#endif
      CK(cudaMemcpy(di, w.items.data(), n * sizeof(Item), cudaMemcpyHostToDevice));
      CK(cudaMemcpy(dp, pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice));
      // launch order of the per-mode sweeps (k_tri, then k_adj_tri), longest first so that the
      // shortest fill the tail: by the number of rows a sweep covers (larger subdomains first),
      // then by mode group (low modes first: the propagating modes carry the complex rows), then
      // item, then column block
      std::vector<int> order;
      for (const Fam f : {F_TRI, F_ATRI}) {
        const int *pt = pre.data() + (size_t)f * (n + 1);
        std::vector<std::array<int, 4>> keys;
        keys.reserve(pt[n]);
        for (int i = 0; i < n; ++i) {
          const SubDesc &d = p->subs[w.items[i].sub].d;
          const int cb = (w.items[i].ncols + 31) / 32, rows = f == F_TRI ? d.NYf : d.Nt;
          for (int l = 0; l < pt[i + 1] - pt[i]; ++l) keys.push_back({-rows, l / cb, i, l});
        }
        std::stable_sort(keys.begin(), keys.end());
        for (const auto &k : keys) order.push_back(pt[k[2]] + k[3]);
      }
      int *dord = nullptr;
      if (!al((void **)&dord, order.size() * sizeof(int))) return MDP_ERR_NOMEM;
      p->d_order[sc].push_back(dord);
      if (!order.empty()) CK(cudaMemcpy(dord, order.data(), order.size() * sizeof(int), cudaMemcpyHostToDevice));
      hpre.push_back(pre);
    }
  }
  return MDP_OK;
}

void wave_batches(const mdp_plan *p, size_t w, Batch *fb, int sc) {
  const int n = (int)p->sched[sc][w].items.size();
  for (int f = 0; f < NFAM; ++f) {
    Batch &b = fb[f];
    std::memset(&b, 0, sizeof b);
    b.items = p->d_items[sc][w];
    b.prefix = p->d_prefix[sc][w] + (size_t)f * (n + 1);
    b.order = f == F_TRI ? p->d_order[sc][w]
              : f == F_ATRI ? p->d_order[sc][w] + p->h_prefix[sc][w][(size_t)F_TRI * (n + 1) + n]
                            : nullptr;
    b.n_items = n;
    b.total_blocks = p->h_prefix[sc][w][(size_t)f * (n + 1) + n];
    set_bounds(p, b, p->out_size, sc == S_GRAD);
  }
}

void single_batches(const mdp_plan *p, const Item &it, Batch *fb, long long out_n) {
  for (int f = 0; f < NFAM; ++f) {
    Batch &b = fb[f];
    std::memset(&b, 0, sizeof b);
    b.items = nullptr;
    b.prefix = nullptr;
    b.n_items = 1;
    b.one = it;
    b.total_blocks = blocks_for((Fam)f, p->subs[it.sub].d, it.ncols);
    set_bounds(p, b, out_n, false);
  }
}

bool device_ok(const mdp_plan *p) { return p && !(p->flags & MDP_PLAN_HOST_ONLY) && p->device >= 0; }

// Around every compute call once a second table set exists: wait for the refactorisation of the
// set in use, and afterwards mark the set as read by work queued on st (chained to its earlier
// readers, so that one event covers them all).
cudaError_t begin_use(const mdp_plan *p, cudaStream_t st) {
  if (!p->ready_ev[p->set]) return cudaSuccess;
  return cudaStreamWaitEvent(st, p->ready_ev[p->set], 0);
}
cudaError_t end_use(mdp_plan *p, cudaStream_t st) {
  if (!p->used_ev[p->set]) return cudaSuccess;
  if (p->used_rec[p->set]) {
    const cudaError_t e = cudaStreamWaitEvent(st, p->used_ev[p->set], 0);
    if (e != cudaSuccess) return e;
  }
  p->used_rec[p->set] = true;
  return cudaEventRecord(p->used_ev[p->set], st);
}
mdp::HostBuf<SubDesc> &stage_of(mdp_plan *p, int set) { return set == 0 ? p->sub_stage : p->alt_stage; }

void destroy_prof(mdp_plan *p) {
  for (int f = 0; f < 16; ++f) {
    for (auto &e : p->prof_ev[f]) { cudaEventDestroy(e.first); cudaEventDestroy(e.second); }
    p->prof_ev[f].clear();
    p->prof_used[f] = 0;
  }
}

}  // namespace

namespace mdp {
void prof_begin(mdp_plan *p, int fam, cudaStream_t st) {
  if (!p->prof_on) return;
  auto &v = p->prof_ev[fam];
  if (p->prof_used[fam] == (int)v.size()) {
    cudaEvent_t a, b;
    if (cudaEventCreate(&a) != cudaSuccess) return;
    if (cudaEventCreate(&b) != cudaSuccess) { cudaEventDestroy(a); return; }
    v.push_back({a, b});
  }
  cudaEventRecord(v[p->prof_used[fam]].first, st);
}
void prof_end(mdp_plan *p, int fam, cudaStream_t st) {
  if (!p->prof_on) return;
  auto &v = p->prof_ev[fam];
  if (p->prof_used[fam] >= (int)v.size()) return;
  cudaEventRecord(v[p->prof_used[fam]].second, st);
  p->prof_used[fam]++;
}
}  // namespace mdp

extern "C" {

const char *mdp_status_string(mdp_status s) {
  switch (s) {
    case MDP_OK: return "ok";
    case MDP_ERR_ARG: return "invalid argument";
    case MDP_ERR_CUDA: return "CUDA error";
    case MDP_ERR_NOMEM: return "out of memory";
    case MDP_ERR_SINGULAR: return "singular tridiagonal system (discrete AP resonance)";
    case MDP_ERR_TIMEOUT: return "device wait timed out";
    case MDP_ERR_STATE: return "call not valid for this plan";
    case MDP_ERR_BOUNDS: return "index out of range (bounds-checked build)";
  }
  return "unknown status";
}

mdp_status mdp_ap_plan(const mdp_subdomain *subs, int n_subs, unsigned flags, mdp_plan **out) {
  return mdp_ap_plan_ex(subs, n_subs, flags, nullptr, out);
}

mdp_status mdp_ap_plan_ex(const mdp_subdomain *subs, int n_subs, unsigned flags, const mdp_plan_options *opt,
                          mdp_plan **out) {
  if (!subs || n_subs < 1 || !out) return MDP_ERR_ARG;
  if (flags & ~(MDP_PLAN_HOST_ONLY | MDP_PLAN_GRAPH | MDP_PLAN_DEDUPE | MDP_PLAN_FP64_COLS | MDP_PLAN_DIRECT_ROWS))
    return MDP_ERR_ARG;
  if (opt && (opt->tile_cols < 0 || opt->workspace_bytes < 0)) return MDP_ERR_ARG;
  if (opt && opt->fft_block_points != 0 &&
      (opt->fft_block_points < FFT_BLOCK_POINTS || opt->fft_block_points > FFT_POINTS ||
       (opt->fft_block_points & (opt->fft_block_points - 1))))
    return MDP_ERR_ARG;
  if (opt && opt->tri_stages != 0 && opt->tri_stages != 2 && opt->tri_stages != 4) return MDP_ERR_ARG;
  *out = nullptr;
  mdp_plan *p = new (std::nothrow) mdp_plan();
  if (!p) return MDP_ERR_NOMEM;
  p->flags = flags;
  p->n_subs = n_subs;
  p->tile_cols = (int)std::max(1LL, env_ll("MDP_TILE_COLS", 256));
  p->ws_budget = env_ll("MDP_WS_MB", 4096) << 20;
  if (opt && opt->tile_cols > 0) p->tile_cols = opt->tile_cols;
  if (opt && opt->workspace_bytes > 0) p->ws_budget = opt->workspace_bytes;
  if (opt && opt->fft_block_points > 0) p->fft_block_points = opt->fft_block_points;
  if (opt && opt->tri_stages > 0) p->tri_stages = opt->tri_stages;
  mdp_status st;
  try {
    st = build_host_plan(p, subs, n_subs);
  } catch (...) {
    st = MDP_ERR_NOMEM;
  }
  if (st == MDP_OK && !(flags & MDP_PLAN_HOST_ONLY)) st = alloc_device(p);
  if (st != MDP_OK) {
    free_device(p);
    delete p;
    return st;
  }
  *out = p;
  return MDP_OK;
}

mdp_status mdp_plan_update_k(mdp_plan *p, const double *k) { return mdp_plan_update_k_stream(p, k, nullptr); }

// Device plans factor on the GPU: the descriptors (new k, stencil coefficients) go up through a
// pinned stage, then one kernel rebuilds every factor, dT/dk and sweep table in place. The host
// copies of the tables are refreshed only when host introspection asks for them.
mdp_status mdp_plan_update_k_stream(mdp_plan *p, const double *k, void *cuda_stream) {
  if (!p || !k) return MDP_ERR_ARG;
  if (!device_ok(p)) return refactor_host(p, k);
  mdp_status st = set_k_fields(p, k);
  if (st != MDP_OK) return st;
  CK(cudaSetDevice(p->device));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  CK(cudaStreamSynchronize(s));   // the stage may still feed an upload of an earlier call
  if (p->ready_ev[p->set]) CK(cudaEventSynchronize(p->ready_ev[p->set]));
  if (p->used_rec[p->set]) CK(cudaStreamWaitEvent(s, p->used_ev[p->set], 0));   // readers on other streams
  HostBuf<SubDesc> &stage = stage_of(p, p->set);
  for (size_t i = 0; i < p->subs.size(); ++i) stage[i] = p->subs[i].d;
  CK(cudaMemcpyAsync(p->d_subs, stage.data(), p->subs.size() * sizeof(SubDesc), cudaMemcpyHostToDevice, s));
  CK(cudaMemsetAsync(p->d_fstatus, 0, sizeof(int), s));
  CK(launch_factor(p, p->d_fstatus, s));
  CK(cudaMemcpyAsync(p->h_fstatus.data(), p->d_fstatus, sizeof(int), cudaMemcpyDeviceToHost, s));
  if (p->ready_ev[p->set]) CK(cudaEventRecord(p->ready_ev[p->set], s));
  CK(cudaStreamSynchronize(s));
  p->host_stale = true;
  return (mdp_status)p->h_fstatus[0];
}

// The refactorisation into the other table set, then the sets swap roles (see include/mdp.h).
mdp_status mdp_plan_update_k_async(mdp_plan *p, const double *k, void *cuda_stream) {
  if (!p || !k) return MDP_ERR_ARG;
  if (!device_ok(p)) return refactor_host(p, k);
  mdp_status st = set_k_fields(p, k);
  if (st != MDP_OK) return st;
  CK(cudaSetDevice(p->device));
  cudaStream_t s = (cudaStream_t)cuda_stream;
  if (!p->alt_tables) {   // first call: the second set starts as a copy of the first (k-independent tables)
    const size_t nt = std::max<size_t>(p->host_tables.size() * sizeof(double), 256);
    const size_t np = std::max<size_t>(p->host_piv.size(), 256);
    const size_t ns = std::max<size_t>(p->subs.size() * sizeof(SubDesc), 256);
    if (cudaMalloc((void **)&p->alt_tables, nt) != cudaSuccess || cudaMalloc((void **)&p->alt_piv, np) != cudaSuccess ||
        cudaMalloc((void **)&p->alt_subs, ns) != cudaSuccess || !p->alt_stage.alloc(p->subs.size(), true))
      return MDP_ERR_NOMEM;
    for (int s_ = 0; s_ < 2; ++s_) {
      CK(cudaEventCreateWithFlags(&p->ready_ev[s_], cudaEventDisableTiming));
      CK(cudaEventCreateWithFlags(&p->used_ev[s_], cudaEventDisableTiming));
    }
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(p->alt_tables, p->d_tables, nt, cudaMemcpyDeviceToDevice));
    CK(cudaMemcpy(p->alt_piv, p->d_piv, np, cudaMemcpyDeviceToDevice));
  }
  const int b = 1 - p->set;
  HostBuf<SubDesc> &stage = stage_of(p, b);
  CK(cudaEventSynchronize(p->ready_ev[b]));   // the stage fed the upload of the last refactorisation into set b
  if (p->used_rec[b]) CK(cudaStreamWaitEvent(s, p->used_ev[b], 0));   // queued calls still reading set b
  for (size_t i = 0; i < p->subs.size(); ++i) stage[i] = p->subs[i].d;
  CK(cudaMemcpyAsync(p->alt_subs, stage.data(), p->subs.size() * sizeof(SubDesc), cudaMemcpyHostToDevice, s));
  CK(launch_factor_to(p, p->alt_subs, p->alt_tables, p->alt_piv, p->d_status, s));
  CK(cudaEventRecord(p->ready_ev[b], s));
  std::swap(p->d_subs, p->alt_subs);
  std::swap(p->d_tables, p->alt_tables);
  std::swap(p->d_piv, p->alt_piv);
  p->set = b;
  p->host_stale = true;
  return MDP_OK;
}

// The host tables are a cache of the device ones for introspection: rebuilt for the current
// wavenumbers after a device refactor.
static mdp_status ensure_host_tables(const mdp_plan *cp) {
  mdp_plan *p = const_cast<mdp_plan *>(cp);
  if (!p->host_stale) return MDP_OK;
  std::vector<double> k;
  for (auto &hs : p->subs) k.push_back(hs.d.k);
  const mdp_status st = refactor_host(p, k.data());
  if (st == MDP_OK) p->host_stale = false;
  return st;
}

long long mdp_plan_update_bytes(const mdp_plan *p) { return p ? (long long)(p->subs.size() * sizeof(SubDesc)) : 0; }

mdp_status mdp_plan_table_sizes(const mdp_plan *p, long long *n_doubles, long long *n_piv) {
  if (!p) return MDP_ERR_ARG;
  if (n_doubles) *n_doubles = (long long)p->host_tables.size();
  if (n_piv) *n_piv = (long long)p->host_piv.size();
  return MDP_OK;
}

mdp_status mdp_plan_table_offsets(const mdp_plan *p, int sub, long long *off) {
  if (!p || !off || sub < 0 || sub >= p->n_subs) return MDP_ERR_ARG;
  const SubDesc &d = p->subs[sub].d;
  off[0] = d.fact_off; off[1] = d.dT_off; off[2] = d.sin_off; off[3] = d.seg_off;
  off[4] = d.fs_off; off[5] = d.geo_off; off[6] = d.piv_off;
  return MDP_OK;
}

mdp_status mdp_plan_read_tables(const mdp_plan *p, int device_side, double *tables, unsigned char *piv) {
  if (!p || !tables || !piv || (device_side != 0 && device_side != 1)) return MDP_ERR_ARG;
  if (device_side) {
    if (!device_ok(p)) return MDP_ERR_STATE;
    CK(cudaSetDevice(p->device));
    CK(cudaDeviceSynchronize());
    CK(cudaMemcpy(tables, p->d_tables, p->host_tables.size() * sizeof(double), cudaMemcpyDeviceToHost));
    CK(cudaMemcpy(piv, p->d_piv, p->host_piv.size(), cudaMemcpyDeviceToHost));
    return MDP_OK;
  }
  const mdp_status st = ensure_host_tables(p);
  if (st != MDP_OK) return st;
  std::memcpy(tables, p->host_tables.data(), p->host_tables.size() * sizeof(double));
  std::memcpy(piv, p->host_piv.data(), p->host_piv.size());
  return MDP_OK;
}

mdp_status mdp_plan_leaders(const mdp_plan *p, int *leader) {
  if (!p || !leader) return MDP_ERR_ARG;
  for (int i = 0; i < p->n_subs; ++i) leader[i] = p->leader[i];
  return MDP_OK;
}

mdp_status mdp_plan_layout(const mdp_plan *p, int sub, int *gamma_size, int *n_cols, long long *out_offset,
                           const int **gamma_nm) {
  if (!p || sub < 0 || sub >= p->n_subs) return MDP_ERR_ARG;
  const HostSub &hs = p->subs[sub];
  if (gamma_size) *gamma_size = hs.d.G;
  if (n_cols) *n_cols = hs.d.n_cols;
  if (out_offset) *out_offset = hs.d.out_off;
  if (gamma_nm) *gamma_nm = hs.gamma_nm.data();
  return MDP_OK;
}

long long mdp_plan_output_size(const mdp_plan *p) { return p ? p->out_size : 0; }

mdp_status mdp_project_batch(mdp_plan *p, const mdp_c64 *xi, mdp_c64 *out, int out_kind, void *cuda_stream) {
  return mdp_project_batch_rec(p, xi, out, nullptr, out_kind, cuda_stream);
}

mdp_status mdp_project_batch_rec(mdp_plan *p, const mdp_c64 *xi, mdp_c64 *out, mdp_c64 *out_rec, int out_kind,
                                 void *cuda_stream) {
  if (!p || !out || (out_kind != MDP_OUT_Q && out_kind != MDP_OUT_P)) return MDP_ERR_ARG;
  if (!device_ok(p)) return MDP_ERR_STATE;
  if (xi && (const void *)xi == (const void *)out) return MDP_ERR_ARG;
  CK(cudaSetDevice(p->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(begin_use(p, st));
  // basis columns without receivers: with duplicates, only the distinct subdomains are solved
  // and their blocks copied to the duplicates
  const bool dedupe = !xi && !out_rec && !p->sched[S_BASIS].empty();
  const int sc = dedupe ? S_BASIS : S_PROJ;
  auto launch_all = [&]() -> cudaError_t {
    for (size_t w = 0; w < p->sched[sc].size(); ++w) {
      Batch fb[NFAM];
      wave_batches(p, w, fb, sc);
      cudaError_t e = launch_project(p, fb, out_kind, (const double2 *)xi, (double2 *)out, (double2 *)out_rec, st);
      if (e != cudaSuccess) return e;
    }
    if (dedupe)
      for (int i = 0; i < p->n_subs; ++i) {
        const int l = p->leader[i];
        if (l == i) continue;
        const SubDesc &d = p->subs[i].d;
        cudaError_t e = cudaMemcpyAsync(out + d.out_off, out + p->subs[l].d.out_off,
                                        (size_t)d.G * d.n_cols * sizeof(mdp_c64), cudaMemcpyDeviceToDevice, st);
        if (e != cudaSuccess) return e;
      }
    return cudaSuccess;
  };
  if (!(p->flags & MDP_PLAN_GRAPH) || st == nullptr) {
    CK(launch_all());
    CK(end_use(p, st));
    return MDP_OK;
  }
  for (auto &g : p->graphs)
    if (g.xi == (const void *)xi && g.out == (void *)out && g.out_rec == (void *)out_rec && g.kind == out_kind &&
        g.st == st && g.tab == p->d_tables) {
      CK(cudaGraphLaunch(g.exec, st));
      CK(end_use(p, st));
      return MDP_OK;
    }
  // capture every launch of this call into one graph
  const bool prof = p->prof_on;
  p->prof_on = false;
  cudaGraph_t graph = nullptr;
  CK(cudaStreamBeginCapture(st, cudaStreamCaptureModeThreadLocal));
  cudaError_t le = launch_all();
  cudaError_t ce = cudaStreamEndCapture(st, &graph);
  p->prof_on = prof;
  if (le != cudaSuccess || ce != cudaSuccess) {
    if (graph) cudaGraphDestroy(graph);
    return MDP_ERR_CUDA;
  }
  cudaGraphExec_t exec = nullptr;
  cudaError_t ie = cudaGraphInstantiate(&exec, graph, 0);
  cudaGraphDestroy(graph);
  if (ie != cudaSuccess) return MDP_ERR_CUDA;
  if (p->graphs.size() >= 8) {
    cudaGraphExecDestroy(p->graphs.front().exec);
    p->graphs.erase(p->graphs.begin());
  }
  p->graphs.push_back({(const void *)xi, (void *)out, (void *)out_rec, out_kind, st, p->d_tables, exec});
  CK(cudaGraphLaunch(exec, st));
  CK(end_use(p, st));
  return MDP_OK;
}

mdp_status mdp_project_columns(mdp_plan *p, int sub, int col0, int ncols, const mdp_c64 *xi, mdp_c64 *out,
                               int out_kind, void *cuda_stream) {
  if (!p || !out || sub < 0 || sub >= p->n_subs || (out_kind != MDP_OUT_Q && out_kind != MDP_OUT_P)) return MDP_ERR_ARG;
  const SubDesc &d = p->subs[sub].d;
  if (col0 < 0 || ncols < 1 || col0 + ncols > d.n_cols) return MDP_ERR_ARG;
  if (!device_ok(p)) return MDP_ERR_STATE;
  CK(cudaSetDevice(p->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(begin_use(p, st));
  for (int c = 0; c < ncols; c += p->tile_cols) {
    Item it;
    std::memset(&it, 0, sizeof it);
    it.sub = sub; it.col0 = col0 + c; it.ncols = std::min(p->tile_cols, ncols - c);
    long long xo, ro, go, yo, ao, so, reo, tot;
    item_workspace(d, it.ncols, false, xo, ro, go, yo, ao, so, reo, tot);
    it.xi_off = xo; it.r_off = ro; it.gr_off = go; it.y_off = yo; it.a_off = ao; it.s_off = so; it.red_off = reo;
    it.io_off = (long long)c * d.G;
    Batch fb[NFAM];
    single_batches(p, it, fb, (long long)ncols * d.G);
    CK(launch_project(p, fb, out_kind, (const double2 *)xi, (double2 *)out, nullptr, st));
  }
  CK(end_use(p, st));
  return MDP_OK;
}

mdp_status mdp_potential(mdp_plan *p, int sub, int ncols, const mdp_c64 *xi, mdp_c64 *u, void *cuda_stream) {
  if (!p || sub < 0 || sub >= p->n_subs || ncols < 1 || !xi || !u) return MDP_ERR_ARG;
  if (!device_ok(p)) return MDP_ERR_STATE;
  if ((const void *)xi == (const void *)u) return MDP_ERR_ARG;
  CK(cudaSetDevice(p->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(begin_use(p, st));
  CK(launch_potential(p, sub, ncols, (const double2 *)xi, (double2 *)u, st));
  CK(end_use(p, st));
  return MDP_OK;
}

mdp_status mdp_source_terms(mdp_plan *p, int sub, const mdp_c64 *f, const mdp_c64 *src4, mdp_c64 *F, mdp_c64 *u,
                            void *cuda_stream) {
  if (!p || sub < 0 || sub >= p->n_subs || !f || !src4 || !F || !u) return MDP_ERR_ARG;
  if ((const void *)f == (const void *)u) return MDP_ERR_ARG;
  if (!device_ok(p)) return MDP_ERR_STATE;
  CK(cudaSetDevice(p->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(begin_use(p, st));
  const cudaError_t e = launch_source_terms(p, sub, (const double2 *)f, (const double2 *)src4, (double2 *)F,
                                            (double2 *)u, st);
  if (e == cudaErrorMemoryAllocation) return MDP_ERR_NOMEM;
  CK(e);
  CK(end_use(p, st));
  return MDP_OK;
}

mdp_status mdp_basis_densities(mdp_plan *p, int sub, int col0, int ncols, mdp_c64 *out, void *cuda_stream) {
  if (!p || sub < 0 || sub >= p->n_subs || !out) return MDP_ERR_ARG;
  const SubDesc &d = p->subs[sub].d;
  if (col0 < 0 || ncols < 1 || col0 + ncols > d.n_cols) return MDP_ERR_ARG;
  if (!device_ok(p)) return MDP_ERR_STATE;
  CK(cudaSetDevice(p->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(begin_use(p, st));
  CK(launch_basis_densities(p, sub, col0, ncols, (double2 *)out, st));
  CK(end_use(p, st));
  return MDP_OK;
}

mdp_status mdp_ap_adjoint(mdp_plan *p, const mdp_c64 *xi, const mdp_c64 *cot, mdp_c64 *grad_xi, double *grad_k,
                          int out_kind, void *cuda_stream) {
  return mdp_ap_adjoint_rec(p, xi, cot, nullptr, grad_xi, grad_k, out_kind, cuda_stream);
}

mdp_status mdp_ap_adjoint_rec(mdp_plan *p, const mdp_c64 *xi, const mdp_c64 *cot, const mdp_c64 *cot_rec,
                              mdp_c64 *grad_xi, double *grad_k, int out_kind, void *cuda_stream) {
  if (!p || !cot || (out_kind != MDP_OUT_Q && out_kind != MDP_OUT_P)) return MDP_ERR_ARG;
  if (!device_ok(p)) return MDP_ERR_STATE;
  if (!grad_xi && !grad_k) return MDP_OK;
  if ((grad_xi && ((const void *)grad_xi == (const void *)cot || (const void *)grad_xi == (const void *)xi)))
    return MDP_ERR_ARG;
  CK(cudaSetDevice(p->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(begin_use(p, st));
  for (size_t w = 0; w < p->sched[S_GRAD].size(); ++w) {
    Batch fb[NFAM];
    wave_batches(p, w, fb, S_GRAD);
    CK(launch_adjoint(p, fb, out_kind, (const double2 *)xi, (const double2 *)cot, (const double2 *)cot_rec,
                      (double2 *)grad_xi, grad_k, st));
  }
  CK(end_use(p, st));
  return MDP_OK;
}

mdp_status mdp_ap_solve_batch(mdp_plan *p, int sub, int nrhs, const mdp_c64 *g, mdp_c64 *u, int adjoint,
                              void *cuda_stream) {
  if (!p || sub < 0 || sub >= p->n_subs || nrhs < 0 || (nrhs > 0 && (!g || !u)) || (adjoint != 0 && adjoint != 1))
    return MDP_ERR_ARG;
  if (!device_ok(p)) return MDP_ERR_STATE;
  if (nrhs == 0) return MDP_OK;
  CK(cudaSetDevice(p->device));
  cudaStream_t st = (cudaStream_t)cuda_stream;
  CK(begin_use(p, st));
  CK(launch_solve(p, sub, nrhs, (const double2 *)g, (double2 *)u, adjoint, st));
  CK(end_use(p, st));
  return MDP_OK;
}

mdp_status mdp_plan_status(mdp_plan *p) {
  if (!p) return MDP_ERR_ARG;
  if (!device_ok(p)) return MDP_OK;
  CK(cudaSetDevice(p->device));
  CK(cudaDeviceSynchronize());
  int s = 0;
  CK(cudaMemcpy(&s, p->d_status, sizeof(int), cudaMemcpyDeviceToHost));
  CK(cudaMemset(p->d_status, 0, sizeof(int)));
  return (mdp_status)s;
}

void mdp_plan_destroy(mdp_plan *p) {
  if (!p) return;
  if (device_ok(p)) {
    for (auto &g : p->graphs) cudaGraphExecDestroy(g.exec);
    p->graphs.clear();
    destroy_prof(p);
    free_device(p);
  }
  delete p;
}

mdp_status mdp_plan_gamma_geometry(const mdp_plan *p, int sub, int *owner, double *rho, double *s) {
  if (!p || sub < 0 || sub >= p->n_subs) return MDP_ERR_ARG;
  const HostSub &hs = p->subs[sub];
  for (int i = 0; i < hs.d.G; ++i) {
    if (owner) owner[i] = hs.owner[i];
    if (rho) rho[i] = hs.rho[i];
    if (s) s[i] = hs.s[i];
  }
  return MDP_OK;
}

mdp_status mdp_host_mode_solve(const mdp_plan *p, int sub, int q, int adjoint, const mdp_c64 *b, mdp_c64 *x) {
  if (!p || sub < 0 || sub >= p->n_subs || !b || !x || (adjoint != 0 && adjoint != 1)) return MDP_ERR_ARG;
  const HostSub &hs = p->subs[sub];
  if (q < 1 || q > hs.d.Nq) return MDP_ERR_ARG;
  const mdp_status st = ensure_host_tables(p);
  if (st != MDP_OK) return st;
  host_mode_solve(hs, q, adjoint, (const double *)b, (double *)x);
  return MDP_OK;
}

mdp_status mdp_plan_profile(mdp_plan *p, int enable) {
  if (!p) return MDP_ERR_ARG;
  if (!device_ok(p)) return MDP_ERR_STATE;
  p->prof_on = enable != 0;
  return MDP_OK;
}

mdp_status mdp_plan_profile_read(mdp_plan *p, int family, double *total_ms, int *launches) {
  if (!p || family < 0 || family >= NFAM) return MDP_ERR_ARG;
  if (!device_ok(p)) return MDP_ERR_STATE;
  double tot = 0.0;
  const int n = p->prof_used[family];
  for (int i = 0; i < n; ++i) {
    auto &e = p->prof_ev[family][i];
    CK(cudaEventSynchronize(e.second));
    float ms = 0.f;
    CK(cudaEventElapsedTime(&ms, e.first, e.second));
    tot += ms;
  }
  p->prof_used[family] = 0;
  if (total_ms) *total_ms = tot;
  if (launches) *launches = n;
  return MDP_OK;
}

mdp_status mdp_plan_set_receivers(mdp_plan *p, const int *rows) {
  if (!p || !rows) return MDP_ERR_ARG;
  for (int i = 0; i < p->n_subs; ++i) {
    const SubDesc &d = p->subs[i].d;
    if (rows[i] != -1 && (rows[i] < d.nlo + 1 || rows[i] > d.nhi - 1)) return MDP_ERR_ARG;
  }
  long long off = 0;
  for (int i = 0; i < p->n_subs; ++i) {
    SubDesc &d = p->subs[i].d;
    d.nrec = rows[i];
    d.rec_off = off;
    if (d.nrec >= 0) off += (long long)d.n_cols * (d.Px - 2);
  }
  p->rec_size = off;
  if (!device_ok(p)) return MDP_OK;
  CK(cudaSetDevice(p->device));
  CK(cudaDeviceSynchronize());
  std::vector<SubDesc> ds;
  for (auto &hs : p->subs) ds.push_back(hs.d);
  CK(cudaMemcpy(p->d_subs, ds.data(), ds.size() * sizeof(SubDesc), cudaMemcpyHostToDevice));
  // the receiver kernel's block counts changed: refresh the prefix sums (same sizes)
  for (int sc = 0; sc < 3; ++sc) {
    auto &waves = p->sched[sc];
    auto &dpre = p->d_prefix[sc];
    auto &hpre = p->h_prefix[sc];
    for (size_t w = 0; w < waves.size(); ++w) {
      const int n = (int)waves[w].items.size();
      auto &pre = hpre[w];
      for (int i = 0; i < n; ++i)
        pre[(size_t)F_IREC * (n + 1) + i + 1] =
            pre[(size_t)F_IREC * (n + 1) + i] + blocks_for(F_IREC, p->subs[waves[w].items[i].sub].d, waves[w].items[i].ncols);
      CK(cudaMemcpy(dpre[w], pre.data(), pre.size() * sizeof(int), cudaMemcpyHostToDevice));
    }
  }
  for (auto &g : p->graphs) cudaGraphExecDestroy(g.exec);
  p->graphs.clear();
  return MDP_OK;
}

mdp_status mdp_plan_receiver_layout(const mdp_plan *p, int sub, int *row, int *m_first, int *count, long long *offset) {
  if (!p || sub < 0 || sub >= p->n_subs) return MDP_ERR_ARG;
  const SubDesc &d = p->subs[sub].d;
  if (row) *row = d.nrec;
  if (m_first) *m_first = d.mlo + 1;
  if (count) *count = d.nrec >= 0 ? d.Px - 2 : 0;
  if (offset) *offset = d.rec_off;
  return MDP_OK;
}

long long mdp_plan_receiver_size(const mdp_plan *p) { return p ? p->rec_size : 0; }

long long mdp_plan_table_bytes(const mdp_plan *p) {
  return p ? (long long)(p->host_tables.size() * sizeof(double) + p->host_piv.size()) : 0;
}

int mdp_kernel_family_count(void) { return NFAM; }

const char *mdp_kernel_family_name(int family) { return fam_name(family); }

mdp_status mdp_plan_sub_info(const mdp_plan *p, int sub, int *info) {
  if (!p || !info || sub < 0 || sub >= p->n_subs) return MDP_ERR_ARG;
  const mdp_status st = ensure_host_tables(p);
  if (st != MDP_OK) return st;
  const HostSub &hs = p->subs[sub];
  const SubDesc &d = hs.d;
  int npiv = 0;
  for (long long i = 0; i < (long long)d.Nq * d.Nt; ++i) npiv += hs.piv[i];
  long long creal = 0;  // complex factor rows swept by the forward projection, over all modes
  for (int q = 0; q < d.Nq; ++q) {
    const int itop = hs.seg[5 * q + 4];
    const int rlo = std::max(hs.seg[5 * q + 2], d.i0), rhi = std::min(std::max(hs.seg[5 * q + 3], rlo), itop);
    creal += (itop - d.i0 + 1) - (rhi - rlo);
  }
  const int vals[14] = {d.Px, d.Py, d.Nq, d.Nt, d.i0, d.nfirst, d.cplx, d.G, d.R, npiv, d.n_cols, d.Nx,
                        d.xsym, (int)creal};
  for (int i = 0; i < 14; ++i) info[i] = vals[i];
  return MDP_OK;
}

}  // extern "C"
