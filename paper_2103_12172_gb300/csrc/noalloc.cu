// mdp_ap_solve_noalloc: the full-grid AP solve of mdp_ap_solve_batch for callers that cannot
// allocate device memory (for example code running where cudaMalloc is unavailable or
// forbidden, such as inside an allocator-free runtime or a caller that owns every device byte).
// Its scratch -- the subdomain descriptor, the per-mode LU factor rows, the sine table, the
// pivot flags (the only tables the full-grid solve reads) and the mode-space buffer -- lives in
// one file-scope device array of fixed size that every GPU loading this library holds until the
// process exits. Nothing is allocated on the device per call.
#include "mdp_internal.h"

#include <algorithm>
#include <cstring>
#include <mutex>

namespace {

constexpr size_t kNoAllocScratchBytes = 32u << 20;  // 32 MiB per device
__device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocScratchBytes];

constexpr int kMaxDevices = 64;
void *g_scratch_addr[kMaxDevices] = {nullptr};
std::mutex g_scratch_mu;

// Device address of the scratch array on the current device. The first call on a device looks
// it up with cudaGetSymbolAddress (the host-side symbol is only a stand-in, not a device address).
mdp_status scratch_address(int dev, void **out) {
  if (dev < 0 || dev >= kMaxDevices) return MDP_ERR_ARG;
  std::lock_guard<std::mutex> lk(g_scratch_mu);
  if (!g_scratch_addr[dev]) {
    void *ptr = nullptr;
    if (cudaGetSymbolAddress(&ptr, g_noalloc_scratch) != cudaSuccess || !ptr) return MDP_ERR_CUDA;
    g_scratch_addr[dev] = ptr;
  }
  *out = g_scratch_addr[dev];
  return MDP_OK;
}

size_t align256(size_t v) { return (v + 255) & ~(size_t)255; }

}  // namespace

extern "C" mdp_status mdp_ap_solve_noalloc(const mdp_subdomain *sub, int nrhs, const mdp_c64 *g, mdp_c64 *u,
                                           int adjoint, void *cuda_stream) {
  if (!sub || nrhs < 0 || (nrhs > 0 && (!g || !u)) || (adjoint != 0 && adjoint != 1)) return MDP_ERR_ARG;
  // host tables for this one subdomain (geometry checks, per-mode factors, sine tables)
  mdp_plan hp;
  hp.flags = MDP_PLAN_HOST_ONLY;
  hp.n_subs = 1;
  mdp_status st;
  try {
    st = mdp::build_host_plan(&hp, sub, 1);
  } catch (...) {
    st = MDP_ERR_NOMEM;
  }
  if (st != MDP_OK) return st;
  const mdp::SubDesc &hs = hp.subs[0].d;
  // scratch layout: [descriptor | factor rows, sine table | pivot flags | mode-space buffer]; the
  // descriptor copied to the device is rebased onto that table (the full-grid solve reads the
  // factor rows, the sines and the pivot flags only, so the other offsets are never followed)
  mdp::SubDesc hd = hs;
  const size_t n_fact = (size_t)hs.Nq * hs.Nt * (hs.cplx ? 8 : 4), n_sin = 4 * (size_t)hs.Nx;
  const size_t n_piv = (size_t)hs.Nq * hs.Nt;
  hd.fact_off = 0;
  hd.sin_off = (long long)((n_fact + 31) & ~(size_t)31);
  hd.piv_off = 0;
  hd.dT_off = hd.geo_off = hd.seg_off = hd.fs_off = hd.tcb_off = 0;
  const size_t off_tab = align256(sizeof(mdp::SubDesc));
  const size_t off_piv = off_tab + align256(((size_t)hd.sin_off + n_sin) * sizeof(double));
  const size_t off_buf = off_piv + align256(n_piv);
  const size_t per_rhs = (size_t)hd.Nq * hd.Nt * 2 * sizeof(double);
  if (off_buf + per_rhs > kNoAllocScratchBytes) return MDP_ERR_ARG;  // grid too large for the fixed scratch
  if (nrhs == 0) return MDP_OK;
  // The descriptor and the host tables are copied from pageable memory that is freed on return:
  // a captured copy node would read freed memory at replay, so a capturing stream is refused
  // before anything is enqueued.
  cudaStream_t s = (cudaStream_t)cuda_stream;
  cudaStreamCaptureStatus cap = cudaStreamCaptureStatusNone;
  if (cudaStreamIsCapturing(s, &cap) != cudaSuccess) return MDP_ERR_CUDA;
  if (cap != cudaStreamCaptureStatusNone) return MDP_ERR_STATE;
  int dev = -1;
  if (cudaGetDevice(&dev) != cudaSuccess) return MDP_ERR_CUDA;
  void *base = nullptr;
  st = scratch_address(dev, &base);
  if (st != MDP_OK) return st;
  unsigned char *b = (unsigned char *)base;
  // pageable-source copies are staged before these calls return, so the host tables may go (and
  // each call waits on the host for the work already queued on `s`)
  if (cudaMemcpyAsync(b, &hd, sizeof hd, cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b + off_tab, hp.host_tables.data() + hs.fact_off, n_fact * sizeof(double),
                      cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b + off_tab + (size_t)hd.sin_off * sizeof(double), hp.host_tables.data() + hs.sin_off,
                      n_sin * sizeof(double), cudaMemcpyHostToDevice, s) != cudaSuccess ||
      cudaMemcpyAsync(b + off_piv, hp.host_piv.data() + hs.piv_off, n_piv, cudaMemcpyHostToDevice, s) != cudaSuccess)
    return MDP_ERR_CUDA;
  const long long buf_doubles = (long long)((kNoAllocScratchBytes - off_buf) / sizeof(double));
  if (mdp::launch_solve_raw((const mdp::SubDesc *)b, hd, (const double *)(b + off_tab), (const uint8_t *)(b + off_piv),
                            (double *)(b + off_buf), buf_doubles, nrhs, (const double2 *)g, (double2 *)u, adjoint,
                            s) != cudaSuccess)
    return MDP_ERR_CUDA;
  return MDP_OK;
}

extern "C" long long mdp_ap_solve_noalloc_limit_bytes(void) { return (long long)kNoAllocScratchBytes; }
