// C ABI of libgpw (declared in include/gpw.h): plan construction and upload, and the
// orchestration of one evaluation on a stream — collocation kernels, cuFFT for the
// level <-> finest-grid Fourier interpolation and the Poisson solve, exchange, and the
// integration / gradient kernels with their fixed-order reductions.
#include <cuda_runtime.h>

#include <array>
#include <map>
#include <memory>
#include <mutex>
#include <cufft.h>

#include <algorithm>
#include <chrono>
#include <thread>
#include <cstring>
#include <memory>
#include <new>
#include <string>
#include <vector>

#include "gpw.h"
#include "gpw_internal.h"
#include "kernels.h"
#include "plan_host.h"

struct gpw_plan_s {
  gpw::Plan p;
};

// A set of plans whose collocation and integration tasks run in single launches.
struct gpw_batch_s {
  int cap = 0, n = 0;
  gpw::PlanView* views = nullptr;       // device, cap entries
  int4* work_c = nullptr;               // merged work lists (device)
  int4* work_i = nullptr;
  long long cap_c = 0, cap_i = 0, nwc = 0, nwi = 0;
  gpw::GridLaunch colloc, integ1;
  std::vector<gpw_plan_t> plans;
  long long generation = 0;             // successful gpw_batch_set calls
};

namespace gpw {

static thread_local std::string g_err;
void set_error(const std::string& msg) { g_err = msg; }

// A cuFFT handle shared by the plans of the process (see fft_entry).
struct FftEntry {
  cufftHandle h;
  size_t ws = 0;
  std::mutex mu;
};

namespace {

#define GPW_CK(x)                                                                   \
  do {                                                                              \
    cudaError_t e_ = (x);                                                           \
    if (e_ != cudaSuccess) {                                                        \
      set_error(std::string(#x) + ": " + cudaGetErrorString(e_));                   \
      return e_ == cudaErrorMemoryAllocation ? GPW_ENOMEM : GPW_ECUDA;              \
    }                                                                               \
  } while (0)

#define GPW_CF(x)                                                                   \
  do {                                                                              \
    cufftResult r_ = (x);                                                           \
    if (r_ != CUFFT_SUCCESS) {                                                      \
      set_error(std::string(#x) + ": cufft error " + std::to_string((int)r_));      \
      return r_ == CUFFT_ALLOC_FAILED ? GPW_ENOMEM : GPW_ECUFFT;                    \
    }                                                                               \
  } while (0)

// Plan memory is stream-ordered (cudaMallocAsync / cudaFreeAsync from the device's
// default pool, kept cached): committing and releasing plans does not synchronise the
// device, so a server can commit and release requests while other batches run.
thread_local cudaStream_t g_alloc_stream = nullptr;  // set by create_device (this thread)

template <class T>
int dalloc(T** ptr, long long count, long long* bytes) {
  size_t b = sizeof(T) * (size_t)std::max<long long>(count, 1);
  GPW_CK(cudaMallocAsync((void**)ptr, b, g_alloc_stream));
  *bytes += (long long)b;
  return GPW_OK;
}

template <class T>
int upload(T** ptr, const std::vector<T>& v, long long* bytes) {
  int rc = dalloc(ptr, (long long)v.size(), bytes);
  if (rc) return rc;
  if (!v.empty())
    GPW_CK(cudaMemcpyAsync(*ptr, v.data(), sizeof(T) * v.size(), cudaMemcpyHostToDevice,
                           g_alloc_stream));
  return GPW_OK;
}

// cuFFT handles shared by all plans of the process, one per (device, mesh, direction),
// made once without a work area (cufftSetAutoAllocation 0).  A plan owns its work area
// and sets it, with its stream, right before each execution under the handle's lock, so
// plans on different streams run the same transform concurrently.
std::mutex g_fft_mu;
std::map<std::array<int, 5>, std::unique_ptr<FftEntry>> g_fft;

int fft_entry(const int* N, cufftType type, FftEntry** out) {
  int dev = 0;
  GPW_CK(cudaGetDevice(&dev));
  std::lock_guard<std::mutex> lk(g_fft_mu);
  const std::array<int, 5> key = {dev, N[0], N[1], N[2], (int)type};
  auto it = g_fft.find(key);
  if (it == g_fft.end()) {
    std::unique_ptr<FftEntry> e(new FftEntry());
    GPW_CF(cufftCreate(&e->h));
    if (cufftSetAutoAllocation(e->h, 0) != CUFFT_SUCCESS ||
        cufftMakePlan3d(e->h, N[0], N[1], N[2], type, &e->ws) != CUFFT_SUCCESS) {
      cufftDestroy(e->h);
      set_error("cufftMakePlan3d failed");
      return GPW_ECUFFT;
    }
    it = g_fft.emplace(key, std::move(e)).first;
  }
  *out = it->second.get();
  return GPW_OK;
}

// cufftEstimate3d per (mesh, direction), remembered (prepare calls it for every plan)
std::map<std::array<int, 4>, size_t> g_fft_est;

size_t fft_estimate(const int* N, cufftType type) {
  std::lock_guard<std::mutex> lk(g_fft_mu);
  const std::array<int, 4> key = {N[0], N[1], N[2], (int)type};
  auto it = g_fft_est.find(key);
  if (it != g_fft_est.end()) return it->second;
  size_t ws = 0;
  if (cufftEstimate3d(N[0], N[1], N[2], type, &ws) != CUFFT_SUCCESS) ws = 0;
  g_fft_est[key] = ws;
  return ws;
}

// Release the plan's device memory in stream order on `stream` (the commit stream if
// NULL); with sync, after all device work so far (the plain destroy's guarantee).
void free_plan(Plan* P, cudaStream_t stream = nullptr, bool sync = true) {
  DeviceArrays& d = P->d;
  void* ptrs[] = {d.hot_a, d.hot_b, d.ids, d.ids2, d.geo, d.cab, d.pref, d.tab_off,
                  d.coef_off, d.part_off, d.xt_off, d.yt_off, d.task_c, d.sub_off_c, d.work_c, d.task_i, d.sub_off_i, d.work_i, d.groups, d.atom_off,
                  d.atom_list, d.tab, d.coef, d.part, d.pgrad, d.grids, d.spec, d.fspec,
                  d.fspec2, d.fine_a, d.fine_b, d.red, d.energies, d.err, d.tabs, d.view, d.g2tab,
                  d.g1tab, d.grad3, d.fspec3, d.mono_t, d.xfer_D, d.xfer_V, d.xfer_g,
                  d.fft_pack, d.fft_tw, P->fft_work};
  bool any = false;
  for (void* q : ptrs) any = any || q != nullptr;
  if (any && sync) cudaDeviceSynchronize();
  cudaStream_t fs = stream ? stream : P->alloc_stream;
  for (void* q : ptrs)
    if (q) cudaFreeAsync(q, fs);
  for (cudaEvent_t e : P->ev_pool) cudaEventDestroy(e);
  P->ev_pool.clear();
  if (P->xfer_ev) cudaEventDestroy(P->xfer_ev);
  if (P->xfer_stream) cudaStreamDestroy(P->xfer_stream);
  P->xfer_ev = nullptr;
  P->xfer_stream = nullptr;
  for (int k = 0; k < GPW_MAX_LEVELS; ++k) P->fft_d2z[k] = P->fft_z2d[k] = P->fft_z2z[k] = nullptr;
  P->fft_work = nullptr;
  d = DeviceArrays();
  recycle_host_arrays(P->host);
  delete P->host;
  P->host = nullptr;
  P->committed = false;
}

// Device bytes create_device will allocate for this plan (cuFFT work areas estimated).
long long estimate_bytes(const Plan& P, const HostArrays& H) {
  auto sz = [](long long n, size_t e) { return (long long)e * std::max<long long>(n, 1); };
  long long b = 0;
  b += sz((long long)H.hot_a.size(), sizeof(int4)) * 4;                 // hot_a, hot_b, ids, ids2
  b += sz((long long)H.geo.size(), sizeof(double)) + sz(P.npairs, sizeof(double)) * 2;
  b += sz(P.npairs, sizeof(long long)) * 5;  // tab, coef, part, xt and yt offsets
  if (P.tasks_on_device) {
    // records and offsets are sized by the counts; the work lists by their bound (a
    // sub-box holds at most one collocation item and 1 + tasks / chunk integration items)
    b += sz(2 * P.nent, sizeof(int4)) + sz(2 * P.nent_i, sizeof(int4));
    b += sz(P.nsub_total + 1, sizeof(long long)) + sz(P.nsub_i + 1, sizeof(long long));
    const long long wc = std::min(P.nsub_total, P.nent);
    const long long wi = std::min(P.nsub_i, P.nent_i) + (P.chunk_i > 0 ? P.nent_i / P.chunk_i : 0);
    b += sz(wc, sizeof(int4)) + sz(wi, sizeof(int4));
    // build scratch beyond the part buffer, released after the commit
    b += std::max<long long>(0, task_sort_bytes(P) + 16 * (P.npairs + 1) -
                                    (long long)sizeof(double) * P.part_total);
  } else {
    b += sz((long long)H.task_c.size(), sizeof(int4)) + sz((long long)H.task_i.size(), sizeof(int4));
    b += sz((long long)H.sub_off_c.size(), sizeof(long long)) + sz((long long)H.sub_off_i.size(), sizeof(long long));
    b += sz((long long)H.work_c.size(), sizeof(int4)) + sz((long long)H.work_i.size(), sizeof(int4));
  }
  b += sz((long long)H.groups.size(), sizeof(int4)) + sz((long long)H.atom_off.size(), sizeof(long long));
  b += sz((long long)H.atom_list.size(), sizeof(int));
  b += sz(P.tab_total + P.coef_total + P.part_total + 6 * P.npairs + P.grid_total, sizeof(double));
  b += sz(P.spec_total + 2 * P.fine_spec_n, sizeof(cufftDoubleComplex));
  b += sz(2 * P.fine_n + 2 * 304 + 2, sizeof(double)) + sizeof(int) + sizeof(CoefTables) + sizeof(PlanView);
  b += 2 * sz((long long)P.lev[0].N[0] + P.lev[0].N[1] + P.lev[0].N[2], sizeof(double));
  if (P.xc == GPW_XC_PBE_X)
    b += sz(3 * P.fine_n, sizeof(double)) + sz(P.fine_spec_n, sizeof(cufftDoubleComplex));
  if (P.skew) b += sz((long long)H.mono_t.size(), sizeof(double));
  size_t ws = 0;  // one work area: the largest transform of the plan
  bool packed = false;
  for (int k = 0; k < P.nlev; ++k) {
    ws = std::max(ws, std::max(fft_estimate(P.lev[k].N, CUFFT_D2Z), fft_estimate(P.lev[k].N, CUFFT_Z2D)));
    if (P.lev[k].N[2] % 2 == 0) {
      const int h[3] = {P.lev[k].N[0], P.lev[k].N[1], P.lev[k].N[2] / 2};
      ws = std::max(ws, fft_estimate(h, CUFFT_Z2Z));
      packed = true;
    }
  }
  b += (long long)ws;
  if (packed) {
    b += sz(P.fine_n / 2, sizeof(cufftDoubleComplex));  // the half-length grid
    long long ntw = 0;
    for (int k = 0; k < P.nlev; ++k) ntw += P.lev[k].N[2] / 2 + 1;
    b += sz(ntw, sizeof(cufftDoubleComplex));           // its twiddles
  }
  return b;
}

int create_device(Plan* P, HostArrays& H, cudaStream_t s) {
  long long b = 0;
  DeviceArrays& d = P->d;
  int rc;
  {
    // keep freed plan memory in the default pool for the next plans
    int dev = 0;
    cudaMemPool_t pool;
    if (cudaGetDevice(&dev) == cudaSuccess && cudaDeviceGetDefaultMemPool(&pool, dev) == cudaSuccess) {
      unsigned long long thr = ~0ULL;
      cudaMemPoolSetAttribute(pool, cudaMemPoolAttrReleaseThreshold, &thr);
    }
  }
  P->alloc_stream = s;
  g_alloc_stream = s;
#define GPW_TRY(x) \
  if ((rc = (x)) != GPW_OK) return rc
  GPW_TRY(upload(&d.hot_a, H.hot_a, &b));
  GPW_TRY(upload(&d.hot_b, H.hot_b, &b));
  GPW_TRY(upload(&d.ids, H.ids, &b));
  GPW_TRY(upload(&d.ids2, H.ids2, &b));
  GPW_TRY(upload(&d.geo, H.geo, &b));
  GPW_TRY(upload(&d.cab, H.cab, &b));
  GPW_TRY(dalloc(&d.pref, P->npairs, &b));
  GPW_TRY(upload(&d.tab_off, H.tab_off, &b));
  GPW_TRY(upload(&d.coef_off, H.coef_off, &b));
  GPW_TRY(upload(&d.part_off, H.part_off, &b));
  GPW_TRY(upload(&d.xt_off, H.xt_off, &b));
  GPW_TRY(upload(&d.yt_off, H.yt_off, &b));
  if (!P->tasks_on_device) {
    GPW_TRY(upload(&d.task_c, H.task_c, &b));
    GPW_TRY(upload(&d.sub_off_c, H.sub_off_c, &b));
    GPW_TRY(upload(&d.work_c, H.work_c, &b));
    GPW_TRY(upload(&d.task_i, H.task_i, &b));
    GPW_TRY(upload(&d.sub_off_i, H.sub_off_i, &b));
    GPW_TRY(upload(&d.work_i, H.work_i, &b));
  }
  GPW_TRY(upload(&d.groups, H.groups, &b));
  GPW_TRY(upload(&d.atom_off, H.atom_off, &b));
  GPW_TRY(upload(&d.atom_list, H.atom_list, &b));
  GPW_TRY(dalloc(&d.tab, P->tab_total, &b));
  GPW_TRY(dalloc(&d.coef, P->coef_total, &b));
  GPW_TRY(dalloc(&d.part, P->part_total, &b));
  GPW_TRY(dalloc(&d.pgrad, 6 * P->npairs, &b));
  GPW_TRY(dalloc(&d.grids, P->grid_total, &b));
  GPW_TRY(dalloc(&d.spec, P->spec_total, &b));
  GPW_TRY(dalloc(&d.fspec, P->fine_spec_n, &b));
  GPW_TRY(dalloc(&d.fspec2, P->fine_spec_n, &b));
  GPW_TRY(dalloc(&d.fine_a, P->fine_n, &b));
  GPW_TRY(dalloc(&d.fine_b, P->fine_n, &b));
  GPW_TRY(dalloc(&d.red, 2 * kRedBlocks, &b));
  // device-built task lists (they may use the part buffer as scratch)
  if (P->tasks_on_device) GPW_TRY(build_tasks_device(P, H, s, &b));
  {
    // ((2 pi s)/L_d)^2 per finest-mesh index along each axis, s the signed frequency,
    // formed as (2 pi s)/L, then squared, as the oracle forms it
    const LevelInfo& f = P->lev[0];
    std::vector<double> g2(f.N[0] + f.N[1] + f.N[2]);
    int o = 0;
    for (int dd = 0; dd < 3; ++dd) {
      // non-orthogonal cell: (2 pi s |b_d|)^2, the cross terms are added by the kernels
      const double bl = std::sqrt(P->rec[3 * dd] * P->rec[3 * dd] + P->rec[3 * dd + 1] * P->rec[3 * dd + 1] +
                                  P->rec[3 * dd + 2] * P->rec[3 * dd + 2]);
      for (int m = 0; m < f.N[dd]; ++m) {
        const int sf = m < (f.N[dd] + 1) / 2 ? m : m - f.N[dd];
        const double g = P->skew ? 2.0 * M_PI * (double)sf * bl : 2.0 * M_PI * (double)sf / P->L[dd];
        g2[o++] = g * g;
      }
    }
    GPW_TRY(upload(&d.g2tab, g2, &b));
    // signed (2 pi s)/L_d for the Fourier derivative, 0 on an even axis' Nyquist plane
    std::vector<double> g1(g2.size());
    o = 0;
    for (int dd = 0; dd < 3; ++dd)
      for (int m = 0; m < f.N[dd]; ++m) {
        const int sf = m < (f.N[dd] + 1) / 2 ? m : m - f.N[dd];
        g1[o++] = (f.N[dd] % 2 == 0 && 2 * m == f.N[dd])
                      ? 0.0
                      : (P->skew ? 2.0 * M_PI * (double)sf : 2.0 * M_PI * (double)sf / P->L[dd]);
      }
    GPW_TRY(upload(&d.g1tab, g1, &b));
  }
  if (P->xc == GPW_XC_PBE_X) {
    GPW_TRY(dalloc(&d.grad3, 3 * P->fine_n, &b));
    GPW_TRY(dalloc(&d.fspec3, P->fine_spec_n, &b));
  }
  if (P->skew) GPW_TRY(upload(&d.mono_t, H.mono_t, &b));
  GPW_TRY(dalloc(&d.energies, 2, &b));
  GPW_TRY(dalloc(&d.err, 1, &b));
  GPW_CK(cudaMemsetAsync(d.err, 0, sizeof(int), s));
  {
    CoefTables t;
    build_coef_tables(&t);
    std::vector<CoefTables> v(1, t);
    GPW_TRY(upload(&d.tabs, v, &b));
  }
#undef GPW_TRY
#define GPW_TRY2(x) \
  if ((rc = (x)) != GPW_OK) return rc
  size_t fws = 0;
  std::vector<cufftDoubleComplex> tw;
  for (int k = 0; k < P->nlev; ++k) {
    const LevelInfo& lv = P->lev[k];
    GPW_TRY2(fft_entry(lv.N, CUFFT_D2Z, &P->fft_d2z[k]));
    GPW_TRY2(fft_entry(lv.N, CUFFT_Z2D, &P->fft_z2d[k]));
    fws = std::max(fws, std::max(P->fft_d2z[k]->ws, P->fft_z2d[k]->ws));
    if (lv.N[2] % 2 == 0) {
      const int h[3] = {lv.N[0], lv.N[1], lv.N[2] / 2};
      GPW_TRY2(fft_entry(h, CUFFT_Z2Z, &P->fft_z2z[k]));
      fws = std::max(fws, P->fft_z2z[k]->ws);
      if (!d.fft_pack) GPW_TRY2(dalloc(&d.fft_pack, P->fine_n / 2, &b));
      P->tw_off[k] = (long long)tw.size();
      rfft_twiddles(lv.N[2], &tw);
    }
  }
  if (!tw.empty()) GPW_TRY2(upload(&d.fft_tw, tw, &b));
  GPW_TRY2(dalloc(&P->fft_work, (long long)((fws + sizeof(double) - 1) / sizeof(double)), &b));
  {
    std::vector<PlanView> v(1, PlanView());
    P->device_bytes = b;
    GPW_CK(configure_kernels(P));
    v[0] = make_view(*P);
    GPW_TRY2(upload(&d.view, v, &b));
  }
  P->work_c_host = H.work_c;
  P->work_i_host = H.work_i;
  P->device_bytes = b;
  GPW_CK(launch_tables(*P, s));
  GPW_CK(launch_validate_tasks(*P, false, s));  // GPW_DEBUG_CHECKS only
  GPW_CK(launch_validate_tasks(*P, true, s));
  // the plan is complete for every stream when the commit returns
  GPW_CK(cudaStreamSynchronize(s));
  P->committed = true;
  return GPW_OK;
}
#undef GPW_TRY2

// Real transforms of level k (unnormalised, cuFFT's conventions).  With an even N2 and a
// 16-byte aligned real grid they run as the complex transform of N0 x N1 x N2/2 plus one
// pass that untangles (forward) or packs (inverse) the half spectrum (rfft.cu); the real
// input of the forward transform and the half spectrum of the inverse stay unchanged.
bool packed(const Plan& P, int k, const void* real) {
  return P.fft_z2z[k] && P.d.fft_pack && P.d.fft_tw && (reinterpret_cast<uintptr_t>(real) & 15) == 0;
}

int fft_d2z(Plan& P, int k, const double* in, cufftDoubleComplex* out, cudaStream_t s) {
  if (packed(P, k, in)) {
    {
      FftEntry* e = P.fft_z2z[k];
      std::lock_guard<std::mutex> lk(e->mu);
      GPW_CF(cufftSetStream(e->h, s));
      GPW_CF(cufftSetWorkArea(e->h, P.fft_work));
      GPW_CF(cufftExecZ2Z(e->h, reinterpret_cast<cufftDoubleComplex*>(const_cast<double*>(in)),
                          P.d.fft_pack, CUFFT_FORWARD));
    }
    GPW_CK(launch_rfft_untangle(P.d.fft_pack, out, P.d.fft_tw + P.tw_off[k], P.lev[k].N, s));
    ++P.launches;
    return GPW_OK;
  }
  FftEntry* e = P.fft_d2z[k];
  std::lock_guard<std::mutex> lk(e->mu);
  GPW_CF(cufftSetStream(e->h, s));
  GPW_CF(cufftSetWorkArea(e->h, P.fft_work));
  GPW_CF(cufftExecD2Z(e->h, const_cast<double*>(in), out));
  return GPW_OK;
}

int fft_z2d(Plan& P, int k, cufftDoubleComplex* in, double* out, cudaStream_t s) {
  if (packed(P, k, out)) {
    GPW_CK(launch_rfft_pack(in, P.d.fft_pack, P.d.fft_tw + P.tw_off[k], P.lev[k].N, s));
    ++P.launches;
    FftEntry* e = P.fft_z2z[k];
    std::lock_guard<std::mutex> lk(e->mu);
    GPW_CF(cufftSetStream(e->h, s));
    GPW_CF(cufftSetWorkArea(e->h, P.fft_work));
    GPW_CF(cufftExecZ2Z(e->h, P.d.fft_pack, reinterpret_cast<cufftDoubleComplex*>(out),
                        CUFFT_INVERSE));
    return GPW_OK;
  }
  FftEntry* e = P.fft_z2d[k];
  std::lock_guard<std::mutex> lk(e->mu);
  GPW_CF(cufftSetStream(e->h, s));
  GPW_CF(cufftSetWorkArea(e->h, P.fft_work));
  GPW_CF(cufftExecZ2D(e->h, in, out));
  return GPW_OK;
}

// Records a CUDA event pair around one phase on the call's stream when profiling.
class Phase {
 public:
  Phase(Plan& P, int ph, cudaStream_t s) : P_(P), s_(s), on_(P.prof) {
    if (!on_) return;
    while (P_.ev_pool.size() < P_.ev_used + 2) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) {
        on_ = false;
        return;
      }
      P_.ev_pool.push_back(e);
    }
    cudaEventRecord(P_.ev_pool[P_.ev_used], s_);
    P_.ev_phase.push_back(ph);
  }
  ~Phase() {
    if (!on_) return;
    cudaEventRecord(P_.ev_pool[P_.ev_used + 1], s_);
    P_.ev_used += 2;
  }

 private:
  Plan& P_;
  cudaStream_t s_;
  bool on_;
};

// Pair D tensors and cleared level grids: everything collocation needs.
int prep_rho(Plan& P, const double* D, cudaStream_t s) {
  {
    Phase ph(P, GPW_PHASE_COEF, s);
    GPW_CK(launch_pair_coef(P, D, s));
    GPW_CK(launch_xcontract(P, s));
  }
  GPW_CK(cudaMemsetAsync(P.d.grids, 0, sizeof(double) * (size_t)P.grid_total, s));
  return GPW_OK;
}

// rho_k on every level (raw collocation, Algorithm 1 / Eq. rho_wrap).
int rho_levels(Plan& P, const double* D, cudaStream_t s) {
  int rc = prep_rho(P, D, s);
  if (rc) return rc;
  Phase ph(P, GPW_PHASE_COLLOCATE, s);
  GPW_CK(launch_collocate(P, s));
  return GPW_OK;
}

// Level densities -> finest spectrum S (Fourier interpolation, Sec. II).
int combine(Plan& P, cudaStream_t s) {
  Phase ph(P, GPW_PHASE_SPECTRAL, s);
  for (int k = 0; k < P.nlev; ++k) {
    int rc = fft_d2z(P, k, P.d.grids + P.lev[k].grid_off, P.d.spec + P.lev[k].spec_off, s);
    if (rc) return rc;
  }
  GPW_CK(launch_combine(P, s));
  return GPW_OK;
}

// Finest-grid potential -> level potentials in P.d.grids (restriction, Sec. II).
int restrict_spectra(Plan& P, const cufftDoubleComplex* fa, const cufftDoubleComplex* fb,
                     cudaStream_t s) {
  for (int k = 0; k < P.nlev; ++k) {
    GPW_CK(launch_restrict(P, k, fa, fb, s));
    int rc = fft_z2d(P, k, P.d.spec + P.lev[k].spec_off, P.d.grids + P.lev[k].grid_off, s);
    if (rc) return rc;
  }
  return GPW_OK;
}

int restrict_levels(Plan& P, const double* v_fine, cudaStream_t s) {
  Phase ph(P, GPW_PHASE_SPECTRAL, s);
  int rc = fft_d2z(P, 0, v_fine, P.d.fspec, s);
  if (rc) return rc;
  for (int k = 0; k < P.nlev; ++k) {
    GPW_CK(launch_restrict(P, k, P.d.fspec, nullptr, s));
    rc = fft_z2d(P, k, P.d.spec + P.lev[k].spec_off, P.d.grids + P.lev[k].grid_off, s);
    if (rc) return rc;
  }
  return GPW_OK;
}

int copy_levels(Plan& P, const double* const* v_levels, cudaStream_t s) {
  for (int k = 0; k < P.nlev; ++k) {
    if (!v_levels[k]) {
      set_error("NULL level potential");
      return GPW_EINVAL;
    }
    const LevelInfo& lv = P.lev[k];
    GPW_CK(cudaMemcpyAsync(P.d.grids + lv.grid_off, v_levels[k],
                           sizeof(double) * (size_t)lv.N[0] * lv.N[1] * lv.N[2],
                           cudaMemcpyDeviceToDevice, s));
  }
  return GPW_OK;
}

// Integration of the level potentials in P.d.grids into V (Algorithm 2, Eq. J_wrap).
int mat_from_grids(Plan& P, double* V, cudaStream_t s) {
  {
    Phase ph(P, GPW_PHASE_INTEGRATE, s);
    GPW_CK(launch_integrate(P, 0, s));
  }
  Phase ph(P, GPW_PHASE_ASSEMBLE, s);
  GPW_CK(launch_reduce_parts(P, 0, s));
  GPW_CK(launch_assemble_V(P, 0, V, s));
  return GPW_OK;
}

// One integration pass at degree L + 1 serves both V (its monomials of degree <= L) and
// the gradient contraction: Algorithms 2 and 3 share the task sweep.

int finish_mat_ip1(Plan& P, const double* D, double* V, double* grad, cudaStream_t s,
                   cudaEvent_t v_ready);

int mat_ip1_from_grids(Plan& P, const double* D, double* V, double* grad, cudaStream_t s,
                       cudaEvent_t v_ready = nullptr) {
  {
    Phase ph(P, GPW_PHASE_INTEGRATE_IP1, s);
    GPW_CK(launch_integrate(P, 1, s));
  }
  return finish_mat_ip1(P, D, V, grad, s, v_ready);
}

// Per-pair V tensors (degree L+1) -> V and, if grad is non-NULL, the gradient; v_ready,
// if given, is recorded on s once V is complete (before the gradient kernels).
int finish_mat_ip1(Plan& P, const double* D, double* V, double* grad, cudaStream_t s,
                   cudaEvent_t v_ready = nullptr) {
  {
    Phase ph(P, GPW_PHASE_ASSEMBLE, s);
    GPW_CK(launch_reduce_parts(P, 1, s));
    GPW_CK(launch_assemble_V(P, 1, V, s));
  }
  if (v_ready) GPW_CK(cudaEventRecord(v_ready, s));
  if (!grad) return GPW_OK;
  Phase ph(P, GPW_PHASE_GRAD, s);
  GPW_CK(launch_grad(P, D, grad, s));
  return GPW_OK;
}

int ip1_from_grids(Plan& P, const double* D, double* grad, cudaStream_t s) {
  {
    Phase ph(P, GPW_PHASE_INTEGRATE_IP1, s);
    GPW_CK(launch_integrate(P, 1, s));
  }
  Phase ph(P, GPW_PHASE_GRAD, s);
  GPW_CK(launch_reduce_parts(P, 1, s));
  GPW_CK(launch_grad(P, D, grad, s));
  return GPW_OK;
}

// Kinetic energy density on every level (meta-GGA): its coefficient tensors (degree L+2),
// their x contraction and the collocation pass with the degree raised by 2.
int tau_levels(Plan& P, const double* D, cudaStream_t s) {
  if (!P.xr) {
    set_error("kinetic-energy-density kernels need a plan built with GPW_TAU");
    return GPW_EINVAL;
  }
  {
    Phase ph(P, GPW_PHASE_COEF, s);
    GPW_CK(launch_pair_coef_tau(P, D, s));
    GPW_CK(launch_xcontract(P, s, 2));
  }
  GPW_CK(cudaMemsetAsync(P.d.grids, 0, sizeof(double) * (size_t)P.grid_total, s));
  Phase ph(P, GPW_PHASE_COLLOCATE, s);
  GPW_CK(launch_collocate(P, s, 2));
  return GPW_OK;
}

// Level potentials of tau in P.d.grids -> (1/2) int v grad phi . grad phi (degree L+2
// V tensors) or, with D, the gradient of <v, tau(D)> (degree L+3).
int mat_tau_from_grids(Plan& P, double* V, cudaStream_t s) {
  if (!P.xr) {
    set_error("kinetic-energy-density kernels need a plan built with GPW_TAU");
    return GPW_EINVAL;
  }
  {
    Phase ph(P, GPW_PHASE_INTEGRATE, s);
    GPW_CK(launch_integrate(P, 2, s));
  }
  Phase ph(P, GPW_PHASE_ASSEMBLE, s);
  GPW_CK(launch_reduce_parts(P, 2, s));
  GPW_CK(launch_assemble_V_tau(P, 2, V, s));
  return GPW_OK;
}

int ip1_tau_from_grids(Plan& P, const double* D, double* grad, cudaStream_t s) {
  if (!P.xr) {
    set_error("kinetic-energy-density kernels need a plan built with GPW_TAU");
    return GPW_EINVAL;
  }
  {
    Phase ph(P, GPW_PHASE_INTEGRATE_IP1, s);
    GPW_CK(launch_integrate(P, 3, s));
  }
  Phase ph(P, GPW_PHASE_GRAD, s);
  GPW_CK(launch_reduce_parts(P, 3, s));
  GPW_CK(launch_grad_tau(P, D, grad, s));
  return GPW_OK;
}

// rho -> interpolation -> Poisson + exchange -> restricted level potentials in P.d.grids;
// energies to energies_dev.  Without v_out the Hartree part stays in G space: each level
// spectrum is mask_k (FFT(v_x)/N + 4 pi S/G^2), one finest-grid C2R fewer.
// GGA exchange (GPW_XC_PBE_X) after rho(r) is on the finest grid, with fspec = S(G):
//   grad_d rho = F^-1(i G_d S); fspec <- v_H(G); e, de/drho, w = 2 de/dsigma grad rho;
//   fa = F(de/drho) - sum_d i G_d F(w_d) (unnormalised), fb = v_H(G): each level keeps
//   fa/N + fb inside its sphere.  Three more inverse and three more forward transforms
//   of the finest grid than LDA exchange.
int gga_potential(Plan& P, const double* rho, double* energies_dev, double* v_out,
                  cudaStream_t s) {
  int rc;
  const long long n = P.fine_n;
  for (int d = 0; d < 3; ++d) {
    GPW_CK(launch_fourier_deriv(P, d, P.d.fspec, P.d.fspec2, false, s));
    if ((rc = fft_z2d(P, 0, P.d.fspec2, P.d.grad3 + d * n, s))) return rc;
  }
  GPW_CK(launch_poisson(P, s));  // fspec <- 4 pi S / G^2, E_H
  GPW_CK(launch_pbe_x(P, rho, P.d.grad3, P.d.fine_a, s));
  GPW_CK(launch_energy_final(P, 0, kRedBlocks, s));
  GPW_CK(launch_energy_final(P, 1, kRedBlocks, s));
  if (energies_dev != P.d.energies)
    GPW_CK(cudaMemcpyAsync(energies_dev, P.d.energies, 2 * sizeof(double),
                           cudaMemcpyDeviceToDevice, s));
  if ((rc = fft_d2z(P, 0, P.d.fine_a, P.d.fspec2, s))) return rc;  // F(de/drho)
  for (int d = 0; d < 3; ++d) {
    if ((rc = fft_d2z(P, 0, P.d.grad3 + d * n, P.d.fspec3, s))) return rc;
    GPW_CK(launch_fourier_deriv(P, d, P.d.fspec3, P.d.fspec2, true, s));  // -= i G_d F(w_d)
  }
  if (v_out) {
    GPW_CK(launch_spec_combine(P, P.d.fspec2, P.d.fspec, P.d.fspec3, s));
    if ((rc = fft_z2d(P, 0, P.d.fspec3, v_out, s))) return rc;
  }
  return restrict_spectra(P, P.d.fspec2, P.d.fspec, s);
}

int potential_from_levels(Plan& P, double* energies_dev, double* rho_out, double* v_out,
                          cudaStream_t s) {
  int rc = combine(P, s);
  if (rc) return rc;
  double* rho = rho_out ? rho_out : P.d.fine_b;
  Phase ph(P, GPW_PHASE_SPECTRAL, s);
  GPW_CK(cudaMemcpyAsync(P.d.fspec2, P.d.fspec, sizeof(cufftDoubleComplex) * (size_t)P.fine_spec_n,
                         cudaMemcpyDeviceToDevice, s));
  if ((rc = fft_z2d(P, 0, P.d.fspec2, rho, s))) return rc;
  if (P.xc == GPW_XC_PBE_X) return gga_potential(P, rho, energies_dev, v_out, s);
  GPW_CK(launch_poisson(P, s));  // fspec <- 4 pi S / G^2, E_H
  if (v_out) {
    GPW_CK(cudaMemcpyAsync(P.d.fspec2, P.d.fspec,
                           sizeof(cufftDoubleComplex) * (size_t)P.fine_spec_n,
                           cudaMemcpyDeviceToDevice, s));
    if ((rc = fft_z2d(P, 0, P.d.fspec2, P.d.fine_a, s))) return rc;  // v_H(r)
    GPW_CK(launch_lda(P, rho, P.d.fine_a, v_out, s));               // v_out = v_H + v_x
  } else {
    GPW_CK(launch_lda(P, rho, nullptr, P.d.fine_a, s));              // v_x only
  }
  GPW_CK(launch_energy_final(P, 0, kRedBlocks, s));
  GPW_CK(launch_energy_final(P, 1, kRedBlocks, s));
  if (energies_dev != P.d.energies)
    GPW_CK(cudaMemcpyAsync(energies_dev, P.d.energies, 2 * sizeof(double),
                           cudaMemcpyDeviceToDevice, s));
  if (v_out) {
    if ((rc = fft_d2z(P, 0, v_out, P.d.fspec, s))) return rc;
    return restrict_spectra(P, P.d.fspec, nullptr, s);
  }
  if ((rc = fft_d2z(P, 0, P.d.fine_a, P.d.fspec2, s))) return rc;   // FFT(v_x)
  return restrict_spectra(P, P.d.fspec2, P.d.fspec, s);
}

int fock_potential(Plan& P, const double* D, double* energies_dev, double* rho_out,
                   double* v_out, cudaStream_t s) {
  int rc = rho_levels(P, D, s);
  if (rc) return rc;
  return potential_from_levels(P, energies_dev, rho_out, v_out, s);
}

// GPW_DEBUG_CHECKS: outputs that are not finite set code 16 of the error word
int check_outputs(Plan& P, cudaStream_t s, const double* a, long long na,
                  const double* b = nullptr, long long nb = 0, const double* c = nullptr,
                  long long nc = 0) {
  if (!P.debug) return GPW_OK;
  GPW_CK(launch_finite_check(P, a, na, s));
  GPW_CK(launch_finite_check(P, b, nb, s));
  GPW_CK(launch_finite_check(P, c, nc, s));
  return GPW_OK;
}

int fock_async(Plan& P, const double* D, double* V, double* energies_dev, double* rho_out,
               double* v_out, cudaStream_t s) {
  int rc = fock_potential(P, D, energies_dev, rho_out, v_out, s);
  if (rc) return rc;
  if ((rc = mat_from_grids(P, V, s))) return rc;
  return check_outputs(P, s, V, (long long)P.nao * P.nao, P.d.energies, 2, rho_out,
                       rho_out ? P.fine_n : 0);
}

int fock_grad_async(Plan& P, const double* D, double* V, double* grad, double* energies_dev,
                    cudaStream_t s, cudaEvent_t v_ready = nullptr) {
  int rc = fock_potential(P, D, energies_dev, nullptr, nullptr, s);
  if (rc) return rc;
  if ((rc = mat_ip1_from_grids(P, D, V, grad, s, v_ready))) return rc;
  return check_outputs(P, s, V, (long long)P.nao * P.nao, grad, 3LL * P.natm, P.d.energies, 2);
}

bool bad(gpw_plan_t plan) {
  if (!plan) {
    set_error("NULL plan");
    return true;
  }
  if (!plan->p.committed) {
    set_error("plan not committed (gpw_plan_commit)");
    return true;
  }
  return false;
}

bool null_plan(gpw_plan_t plan) {
  if (!plan) {
    set_error("NULL plan");
    return true;
  }
  return false;
}

}  // namespace
}  // namespace gpw

using gpw::set_error;

extern "C" {

int gpw_plan_prepare(const gpw_desc* desc, gpw_plan_t* out) {
  if (!out) {
    set_error("gpw_plan_prepare: NULL out");
    return GPW_EINVAL;
  }
  try {
    std::unique_ptr<gpw_plan_s> h(new gpw_plan_s());
    std::unique_ptr<gpw::HostArrays> H(new gpw::HostArrays());
    int rc = gpw::build_host_plan(desc, &h->p, H.get());
    if (rc) return rc;
    h->p.device_bytes = gpw::estimate_bytes(h->p, *H);
    h->p.host = H.release();
    *out = h.release();
    return GPW_OK;
  } catch (const std::bad_alloc&) {
    set_error("gpw_plan_prepare: host allocation failed");
    return GPW_ENOMEM;
  } catch (...) {
    set_error("gpw_plan_prepare: unexpected exception");
    return GPW_EINVAL;
  }
}

int gpw_plan_commit(gpw_plan_t plan, void* stream) {
  if (gpw::null_plan(plan)) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  if (P.committed) return GPW_OK;
  if (!P.host) {
    set_error("gpw_plan_commit: plan has no host data");
    return GPW_EINVAL;
  }
  try {
    cudaGetDevice(&P.device);
    int rc = gpw::create_device(&P, *P.host, (cudaStream_t)stream);
    if (rc) {
      // release what was allocated; the host data stays so the commit can be retried
      gpw::HostArrays* keep = P.host;
      P.host = nullptr;
      gpw::free_plan(&P);
      P.host = keep;
      return rc;
    }
    gpw::recycle_host_arrays(P.host);
    delete P.host;
    P.host = nullptr;
    return GPW_OK;
  } catch (const std::bad_alloc&) {
    set_error("gpw_plan_commit: host allocation failed");
    return GPW_ENOMEM;
  }
}

int gpw_plan(const gpw_desc* desc, void* stream, gpw_plan_t* out) {
  if (!out) {
    set_error("gpw_plan: NULL out");
    return GPW_EINVAL;
  }
  gpw_plan_t h = nullptr;
  int rc = gpw_plan_prepare(desc, &h);
  if (rc) return rc;
  rc = gpw_plan_commit(h, stream);
  if (rc) {
    gpw_plan_destroy(h);
    return rc;
  }
  *out = h;
  return GPW_OK;
}

int gpw_plan_query(gpw_plan_t plan, gpw_plan_info* info) {
  if (gpw::null_plan(plan) || !info) return GPW_EINVAL;
  const gpw::Plan& P = plan->p;
  std::memset(info, 0, sizeof(*info));
  info->nao = P.nao;
  info->natm = P.natm;
  info->nlevels = P.nlev;
  info->lmax = P.lmax;
  for (int k = 0; k < P.nlev; ++k) {
    for (int d = 0; d < 3; ++d) info->meshes[k][d] = P.lev[k].N[d];
    info->level_cutoff[k] = P.E[k];
    info->npairs_level[k] = P.npairs_level[k];
    info->pair_points_level[k] = P.pair_points_level[k];
  }
  for (int l = 0; l < 8; ++l) info->pair_points_L[l] = P.pair_points_L[l];
  info->npairs = P.npairs;
  info->pair_points = P.pair_points;
  info->nentries = P.nent;
  info->device_bytes = P.device_bytes;
  info->flops_rho = P.flops_rho;
  info->flops_mat = P.flops_mat;
  info->flops_ip1 = P.flops_ip1;
  info->tile[0] = P.tile[0];
  info->tile[1] = P.tile[1];
  info->tile[2] = P.tile[2];
  for (int d = 0; d < 3; ++d) info->tile_integ[d] = P.tile_i[d];
  info->integ_zwin = P.zwin_i;
  info->nentries_integ = P.nent_i;
  info->colloc_warps = P.committed ? P.nw_colloc : 0;
  info->integ_chunk = P.chunk_i;
  info->xc = P.xc;
  info->volume = P.omega;
  for (int k = 0; k < P.nlev; ++k) info->weight[k] = P.lev[k].weight;
  return GPW_OK;
}

int gpw_plan_update_coords(gpw_plan_t plan, const double* coords, void* stream) {
  if (gpw::bad(plan) || !coords) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  const long long np = P.npairs;
  std::vector<double> geo(8 * np);
  for (long long p = 0; p < np; ++p) {
    const int a = P.pair_a[p], b = P.pair_b[p];
    const int ia = P.prim_atom[a], ib = P.prim_atom[b];
    for (int d = 0; d < 3; ++d) {
      geo[8 * p + d] = coords[3 * ia + d];
      geo[8 * p + 3 + d] =
          P.skew ? coords[3 * ib + d] + (((double)P.h_img[3 * p] * P.lat[d] +
                                           (double)P.h_img[3 * p + 1] * P.lat[3 + d]) +
                                          (double)P.h_img[3 * p + 2] * P.lat[6 + d])
                 : coords[3 * ib + d] + (double)P.h_img[3 * p + d] * P.L[d];
    }
    geo[8 * p + 6] = P.prim_alpha[a];
    geo[8 * p + 7] = P.prim_alpha[b];
  }
  cudaStream_t s = (cudaStream_t)stream;
  if (np) {
    cudaError_t e = cudaMemcpyAsync(P.d.geo, geo.data(), sizeof(double) * geo.size(),
                                    cudaMemcpyHostToDevice, s);
    if (e == cudaSuccess) e = cudaStreamSynchronize(s);
    if (e != cudaSuccess) {
      set_error(std::string("update_coords: ") + cudaGetErrorString(e));
      return GPW_ECUDA;
    }
  }
  P.coords.assign(coords, coords + 3 * P.natm);
  cudaError_t e = gpw::launch_tables(P, s);
  if (e != cudaSuccess) {
    set_error(std::string("update_coords: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  return GPW_OK;
}

int gpw_plan_pairs(gpw_plan_t plan, int* ab, int* img, int* level, int* lo, int* hi) {
  if (gpw::null_plan(plan)) return GPW_EINVAL;
  const gpw::Plan& P = plan->p;
  if (ab) std::copy(P.h_ab.begin(), P.h_ab.end(), ab);
  if (img) std::copy(P.h_img.begin(), P.h_img.end(), img);
  if (level) std::copy(P.h_lev.begin(), P.h_lev.end(), level);
  if (lo) std::copy(P.h_lo.begin(), P.h_lo.end(), lo);
  if (hi) std::copy(P.h_hi.begin(), P.h_hi.end(), hi);
  return GPW_OK;
}

int gpw_plan_task_lists(gpw_plan_t plan, int integ, long long* nent, long long* nsub,
                        long long* nwork, int* tasks, long long* sub_off, int* work) {
  if (gpw::bad(plan) || !nent || !nsub || !nwork || (integ != 0 && integ != 1)) {
    if (plan && plan->p.committed) set_error("gpw_plan_task_lists: bad arguments");
    return GPW_EINVAL;
  }
  const gpw::Plan& P = plan->p;
  *nent = integ ? P.nent_i : P.nent;
  *nsub = integ ? P.nsub_i : P.nsub_total;
  *nwork = integ ? P.nwork_i : P.nwork;
  cudaError_t e = cudaDeviceSynchronize();
  if (e == cudaSuccess && tasks && *nent)
    e = cudaMemcpy(tasks, integ ? P.d.task_i : P.d.task_c, sizeof(int4) * 2 * (size_t)*nent,
                   cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && sub_off)
    e = cudaMemcpy(sub_off, integ ? P.d.sub_off_i : P.d.sub_off_c,
                   sizeof(long long) * (size_t)(*nsub + 1), cudaMemcpyDeviceToHost);
  if (e == cudaSuccess && work && *nwork)
    e = cudaMemcpy(work, integ ? P.d.work_i : P.d.work_c, sizeof(int4) * (size_t)*nwork,
                   cudaMemcpyDeviceToHost);
  if (e != cudaSuccess) {
    set_error(std::string("gpw_plan_task_lists: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  return GPW_OK;
}

int gpw_eval_rho_levels(gpw_plan_t plan, const double* D, double* const* rho_levels,
                        void* stream) {
  if (gpw::bad(plan) || !D || !rho_levels) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::rho_levels(P, D, s);
  if (rc) return rc;
  for (int k = 0; k < P.nlev; ++k) {
    if (!rho_levels[k]) continue;
    const gpw::LevelInfo& lv = P.lev[k];
    cudaError_t e = cudaMemcpyAsync(rho_levels[k], P.d.grids + lv.grid_off,
                                    sizeof(double) * (size_t)lv.N[0] * lv.N[1] * lv.N[2],
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      set_error(std::string("eval_rho_levels: ") + cudaGetErrorString(e));
      return GPW_ECUDA;
    }
  }
  return GPW_OK;
}

int gpw_eval_rho(gpw_plan_t plan, const double* D, double* rho_fine, void* stream) {
  if (gpw::bad(plan) || !D || !rho_fine) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::rho_levels(P, D, s);
  if (rc) return rc;
  if ((rc = gpw::combine(P, s))) return rc;
  if ((rc = gpw::fft_z2d(P, 0, P.d.fspec, rho_fine, s))) return rc;
  return gpw::check_outputs(P, s, rho_fine, P.fine_n);
}

int gpw_eval_mat(gpw_plan_t plan, const double* v_fine, double* V, void* stream) {
  if (gpw::bad(plan) || !v_fine || !V) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::restrict_levels(P, v_fine, s);
  if (rc) return rc;
  if ((rc = gpw::mat_from_grids(P, V, s))) return rc;
  return gpw::check_outputs(P, s, V, (long long)P.nao * P.nao);
}

int gpw_eval_mat_levels(gpw_plan_t plan, const double* const* v_levels, double* V,
                        void* stream) {
  if (gpw::bad(plan) || !v_levels || !V) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::copy_levels(P, v_levels, s);
  if (rc) return rc;
  return gpw::mat_from_grids(P, V, s);
}

int gpw_eval_mat_ip1(gpw_plan_t plan, const double* D, const double* v_fine, double* grad,
                     void* stream) {
  if (gpw::bad(plan) || !D || !v_fine || !grad) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::restrict_levels(P, v_fine, s);
  if (rc) return rc;
  if ((rc = gpw::ip1_from_grids(P, D, grad, s))) return rc;
  return gpw::check_outputs(P, s, grad, 3LL * P.natm);
}

int gpw_eval_tau_levels(gpw_plan_t plan, const double* D, double* const* tau_levels,
                        void* stream) {
  if (gpw::bad(plan) || !D || !tau_levels) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::tau_levels(P, D, s);
  if (rc) return rc;
  for (int k = 0; k < P.nlev; ++k) {
    if (!tau_levels[k]) continue;
    const gpw::LevelInfo& lv = P.lev[k];
    cudaError_t e = cudaMemcpyAsync(tau_levels[k], P.d.grids + lv.grid_off,
                                    sizeof(double) * (size_t)lv.N[0] * lv.N[1] * lv.N[2],
                                    cudaMemcpyDeviceToDevice, s);
    if (e != cudaSuccess) {
      set_error(std::string("eval_tau_levels: ") + cudaGetErrorString(e));
      return GPW_ECUDA;
    }
  }
  return GPW_OK;
}
int gpw_eval_tau(gpw_plan_t plan, const double* D, double* tau_fine, void* stream) {
  if (gpw::bad(plan) || !D || !tau_fine) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::tau_levels(P, D, s);
  if (rc) return rc;
  if ((rc = gpw::combine(P, s))) return rc;
  return gpw::fft_z2d(P, 0, P.d.fspec, tau_fine, s);
}
int gpw_eval_mat_tau(gpw_plan_t plan, const double* v_fine, double* V, void* stream) {
  if (gpw::bad(plan) || !v_fine || !V) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::restrict_levels(P, v_fine, s);
  if (rc) return rc;
  return gpw::mat_tau_from_grids(P, V, s);
}
int gpw_eval_mat_tau_levels(gpw_plan_t plan, const double* const* v_levels, double* V,
                            void* stream) {
  if (gpw::bad(plan) || !v_levels || !V) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::copy_levels(P, v_levels, s);
  if (rc) return rc;
  return gpw::mat_tau_from_grids(P, V, s);
}
int gpw_eval_mat_tau_ip1(gpw_plan_t plan, const double* D, const double* v_fine, double* grad,
                         void* stream) {
  if (gpw::bad(plan) || !D || !v_fine || !grad) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::restrict_levels(P, v_fine, s);
  if (rc) return rc;
  return gpw::ip1_tau_from_grids(P, D, grad, s);
}
int gpw_eval_mat_tau_ip1_levels(gpw_plan_t plan, const double* D,
                                const double* const* v_levels, double* grad, void* stream) {
  if (gpw::bad(plan) || !D || !v_levels || !grad) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::copy_levels(P, v_levels, s);
  if (rc) return rc;
  return gpw::ip1_tau_from_grids(P, D, grad, s);
}
int gpw_eval_mat_ip1_levels(gpw_plan_t plan, const double* D, const double* const* v_levels,
                            double* grad, void* stream) {
  if (gpw::bad(plan) || !D || !v_levels || !grad) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::copy_levels(P, v_levels, s);
  if (rc) return rc;
  return gpw::ip1_from_grids(P, D, grad, s);
}

int gpw_fock_async(gpw_plan_t plan, const double* D, double* V, double* energies_dev,
                   double* rho_out, double* v_fine_out, void* stream) {
  if (gpw::bad(plan) || !D || !V || !energies_dev) return GPW_EINVAL;
  return gpw::fock_async(plan->p, D, V, energies_dev, rho_out, v_fine_out, (cudaStream_t)stream);
}

int gpw_fock(gpw_plan_t plan, const double* D, double* V, double* energies, double* rho_out,
             double* v_fine_out, void* stream) {
  if (gpw::bad(plan) || !D || !V || !energies) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::fock_async(P, D, V, P.d.energies, rho_out, v_fine_out, s);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(energies, P.d.energies, 2 * sizeof(double),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("gpw_fock: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  return GPW_OK;
}

int gpw_fock_grad_async(gpw_plan_t plan, const double* D, double* V, double* grad,
                        double* energies_dev, void* stream) {
  if (gpw::bad(plan) || !D || !V || !grad || !energies_dev) return GPW_EINVAL;
  return gpw::fock_grad_async(plan->p, D, V, grad, energies_dev, (cudaStream_t)stream);
}

int gpw_fock_grad(gpw_plan_t plan, const double* D, double* V, double* grad, double* energies,
                  void* stream) {
  if (gpw::bad(plan) || !D || !V || !grad || !energies) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int rc = gpw::fock_grad_async(P, D, V, grad, P.d.energies, s);
  if (rc) return rc;
  cudaError_t e = cudaMemcpyAsync(energies, P.d.energies, 2 * sizeof(double),
                                  cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("gpw_fock_grad: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  return GPW_OK;
}

int gpw_fock_grad_host(gpw_plan_t plan, const double* D, double* V, double* grad,
                       double* energies, void* stream) {
  if (gpw::bad(plan) || !D || !V || !grad || !energies) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  const size_t nn = sizeof(double) * (size_t)P.nao * (size_t)P.nao;
  const size_t ng = sizeof(double) * 3 * (size_t)P.natm;
  cudaError_t e = cudaSuccess;
  if (!P.d.xfer_D) {
    // first call: the plan's device copies of D, V and the gradient, kept with the plan
    e = cudaMallocAsync((void**)&P.d.xfer_D, nn, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&P.d.xfer_V, nn, s);
    if (e == cudaSuccess) e = cudaMallocAsync((void**)&P.d.xfer_g, ng, s);
    if (e != cudaSuccess) {
      set_error(std::string("gpw_fock_grad_host: ") + cudaGetErrorString(e));
      return GPW_ENOMEM;
    }
    P.device_bytes += (long long)(2 * nn + ng);
  }
  if (!P.xfer_stream) {
    e = cudaStreamCreateWithFlags(&P.xfer_stream, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&P.xfer_ev, cudaEventDisableTiming);
    if (e != cudaSuccess) {
      set_error(std::string("gpw_fock_grad_host: ") + cudaGetErrorString(e));
      return GPW_ECUDA;
    }
  }
  e = cudaMemcpyAsync(P.d.xfer_D, D, nn, cudaMemcpyHostToDevice, s);
  if (e != cudaSuccess) {
    set_error(std::string("gpw_fock_grad_host: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  // V goes back on the copy stream as soon as it is assembled, while the gradient
  // kernels run on s
  int rc = gpw::fock_grad_async(P, P.d.xfer_D, P.d.xfer_V, P.d.xfer_g, P.d.energies, s,
                                P.xfer_ev);
  if (rc) return rc;
  e = cudaStreamWaitEvent(P.xfer_stream, P.xfer_ev, 0);
  if (e == cudaSuccess) e = cudaMemcpyAsync(V, P.d.xfer_V, nn, cudaMemcpyDeviceToHost, P.xfer_stream);
  if (e == cudaSuccess) e = cudaMemcpyAsync(grad, P.d.xfer_g, ng, cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(energies, P.d.energies, 2 * sizeof(double), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(P.xfer_stream);
  if (e != cudaSuccess) {
    set_error(std::string("gpw_fock_grad_host: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  return GPW_OK;
}

int gpw_batch_create(int max_plans, gpw_batch_t* out) {
  if (!out || max_plans < 1) {
    set_error("gpw_batch_create: bad arguments");
    return GPW_EINVAL;
  }
  try {
    gpw_batch_s* b = new gpw_batch_s();
    b->cap = max_plans;
    cudaError_t e = cudaMalloc((void**)&b->views, sizeof(gpw::PlanView) * (size_t)max_plans);
    if (e != cudaSuccess) {
      delete b;
      set_error(std::string("gpw_batch_create: ") + cudaGetErrorString(e));
      return GPW_ENOMEM;
    }
    *out = b;
    return GPW_OK;
  } catch (const std::bad_alloc&) {
    set_error("gpw_batch_create: host allocation failed");
    return GPW_ENOMEM;
  }
}

int gpw_batch_set(gpw_batch_t b, int nplans, const gpw_plan_t* plans, void* stream) {
  if (!b || nplans < 1 || nplans > b->cap || !plans) {
    set_error("gpw_batch_set: bad arguments or more plans than the batch capacity");
    return GPW_EINVAL;
  }
  int lmax = 0;
  int skew_kind = 0;  // 1: a plan needs every cross factor, 2: R01 only (kernels' layout)
  for (int i = 0; i < nplans; ++i) {
    if (gpw::bad(plans[i])) return GPW_EINVAL;
    if (plans[i]->p.skew) skew_kind = (plans[i]->p.skew_zc || skew_kind == 1) ? 1 : 2;
    const gpw::Plan& P = plans[i]->p;
    const gpw::Plan& P0 = plans[0]->p;
    for (int d = 0; d < 3; ++d)
      if (P.tile[d] != P0.tile[d] || P.tile_i[d] != P0.tile_i[d] || P.zwin_i != P0.zwin_i) {
        set_error("gpw_batch_set: plans of a batch must share their sub-box shapes");
        return GPW_EINVAL;
      }
    if (P.device != P0.device) {
      set_error("gpw_batch_set: plans of a batch must live on one device");
      return GPW_EINVAL;
    }
    if (P.skew != P0.skew) {
      set_error("gpw_batch_set: a batch holds orthorhombic or non-orthogonal cells, not both");
      return GPW_EINVAL;
    }
    lmax = std::max(lmax, P.lmax);
  }
  cudaError_t e = gpw::configure_batch(plans[0]->p.tile, plans[0]->p.tile_i, plans[0]->p.zwin_i, lmax,
                                       plans[0]->p.nw_colloc_req, &b->colloc,
                                       &b->integ1, skew_kind);
  if (e != cudaSuccess) {
    set_error(std::string("gpw_batch_set: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  // views, and the work lists of all plans merged band by band: every plan's list is
  // cut into runs of kBand consecutive items (Morton-local sub-boxes, heaviest first
  // inside), and the runs of all plans go by decreasing mean tasks per item, so blocks
  // resident together still share their pairs' tables in L2 and light items come last
  std::vector<gpw::PlanView> views(nplans);
  for (int i = 0; i < nplans; ++i) views[i] = gpw::make_view(plans[i]->p);
  auto merge = [&](bool integ) {
    struct Run {
      double mean;
      int plan;
      size_t first, n;
    };
    std::vector<Run> runs;
    size_t total = 0;
    for (int i = 0; i < nplans; ++i) {
      const std::vector<int4>& w = integ ? plans[i]->p.work_i_host : plans[i]->p.work_c_host;
      for (size_t a = 0; a < w.size(); a += (size_t)gpw::kBand) {
        const size_t n = std::min(w.size() - a, (size_t)gpw::kBand);
        double sum = 0;
        for (size_t j = a; j < a + n; ++j) sum += (double)w[j].w;
        runs.push_back({sum / (double)n, i, a, n});
      }
      total += w.size();
    }
    std::stable_sort(runs.begin(), runs.end(),
                     [](const Run& x, const Run& y) { return x.mean > y.mean; });
    std::vector<int4> out;
    out.reserve(total);
    for (const Run& r : runs) {
      const std::vector<int4>& w = integ ? plans[r.plan]->p.work_i_host : plans[r.plan]->p.work_c_host;
      for (size_t j = r.first; j < r.first + r.n; ++j)
        out.push_back(make_int4(r.plan, w[j].y, w[j].z, w[j].w));
    }
    return out;
  };
  const std::vector<int4> wc = merge(false), wi = merge(true);
  cudaStream_t s = (cudaStream_t)stream;
  // grown in stream order on the batch's stream (the previous launch that read the old
  // list was enqueued there), so other streams' work is not waited for
  auto ensure = [&](int4** ptr, long long* cap, size_t n) -> cudaError_t {
    if ((long long)n <= *cap) return cudaSuccess;
    if (*ptr) cudaFreeAsync(*ptr, s);
    *ptr = nullptr;
    *cap = 0;
    const size_t want = std::max<size_t>(n + n / 4, 1);
    cudaError_t r = cudaMallocAsync((void**)ptr, sizeof(int4) * want, s);
    if (r == cudaSuccess) *cap = (long long)want;
    return r;
  };
  e = ensure(&b->work_c, &b->cap_c, wc.size());
  if (e == cudaSuccess) e = ensure(&b->work_i, &b->cap_i, wi.size());
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->views, views.data(), sizeof(gpw::PlanView) * views.size(),
                        cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !wc.empty())
    e = cudaMemcpyAsync(b->work_c, wc.data(), sizeof(int4) * wc.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess && !wi.empty())
    e = cudaMemcpyAsync(b->work_i, wi.data(), sizeof(int4) * wi.size(), cudaMemcpyHostToDevice, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e != cudaSuccess) {
    set_error(std::string("gpw_batch_set: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  b->n = nplans;
  b->nwc = (long long)wc.size();
  b->nwi = (long long)wi.size();
  b->plans.assign(plans, plans + nplans);
  ++b->generation;
  return GPW_OK;
}

int gpw_stream_wait(void* stream, double timeout_s) {
  if (!(timeout_s >= 0.0)) {
    set_error("gpw_stream_wait: timeout must be >= 0");
    return GPW_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const auto t0 = std::chrono::steady_clock::now();
  std::chrono::microseconds nap(20);
  for (;;) {
    const cudaError_t e = cudaStreamQuery(s);
    if (e == cudaSuccess) return GPW_OK;
    if (e != cudaErrorNotReady) {
      set_error(std::string("gpw_stream_wait: ") + cudaGetErrorString(e));
      return GPW_ECUDA;
    }
    const double waited =
        std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count();
    if (waited >= timeout_s) {
      set_error("gpw_stream_wait: the stream's work did not finish within the timeout");
      return GPW_ETIMEDOUT;
    }
    std::this_thread::sleep_for(nap);
    nap = std::min(nap * 2, std::chrono::microseconds(1000));
  }
}

int gpw_batch_generation(gpw_batch_t b, long long* generation) {
  if (!b || !generation) return GPW_EINVAL;
  *generation = b->generation;
  return GPW_OK;
}

int gpw_batch_fock_grad_async(gpw_batch_t b, const double* const* D, double* const* V,
                              double* const* grad, double* energies_dev, void* stream) {
  if (!b || b->n < 1 || !D || !V || !energies_dev) {
    set_error("gpw_batch_fock_grad_async: batch not set or NULL argument");
    return GPW_EINVAL;
  }
  cudaStream_t s = (cudaStream_t)stream;
  const int n = b->n;
  for (int i = 0; i < n; ++i) {
    if (!D[i] || !V[i]) {
      set_error("gpw_batch_fock_grad_async: NULL D or V");
      return GPW_EINVAL;
    }
    int rc = gpw::prep_rho(b->plans[i]->p, D[i], s);
    if (rc) return rc;
  }
  // the batched grid passes are timed on the first plan's phase timers (gpw_profile)
  gpw::Plan& P0 = b->plans[0]->p;
  cudaError_t e;
  {
    gpw::Phase ph(P0, GPW_PHASE_COLLOCATE, s);
    e = gpw::launch_collocate_views(b->colloc, b->views, b->work_c, b->nwc, P0.d.tabs, s);
  }
  if (e != cudaSuccess) {
    set_error(std::string("batch collocation: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  for (int i = 0; i < n; ++i) {
    int rc = gpw::potential_from_levels(b->plans[i]->p, energies_dev + 2 * i, nullptr, nullptr, s);
    if (rc) return rc;
  }
  {
    gpw::Phase ph(P0, GPW_PHASE_INTEGRATE_IP1, s);
    e = gpw::launch_integrate_views(b->integ1, 1, b->views, b->work_i, b->nwi, P0.d.tabs, s);
  }
  if (e != cudaSuccess) {
    set_error(std::string("batch integration: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  for (int i = 0; i < n; ++i) {
    int rc = gpw::finish_mat_ip1(b->plans[i]->p, D[i], V[i], grad ? grad[i] : nullptr, s);
    if (rc) return rc;
  }
  b->plans[0]->p.launches += 2;
  return GPW_OK;
}

void gpw_batch_destroy(gpw_batch_t b) {
  if (!b) return;
  if (b->views) cudaFree(b->views);
  if (b->work_c) cudaFree(b->work_c);
  if (b->work_i) cudaFree(b->work_i);
  delete b;
}

int gpw_check_device(gpw_plan_t plan, int* code, void* stream) {
  if (gpw::bad(plan)) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  cudaStream_t s = (cudaStream_t)stream;
  int h = 0;
  cudaError_t e = cudaMemcpyAsync(&h, P.d.err, sizeof(int), cudaMemcpyDeviceToHost, s);
  if (e == cudaSuccess) e = cudaStreamSynchronize(s);
  if (e == cudaSuccess) e = cudaMemsetAsync(P.d.err, 0, sizeof(int), s);
  if (e != cudaSuccess) {
    set_error(std::string("gpw_check_device: ") + cudaGetErrorString(e));
    return GPW_ECUDA;
  }
  if (code) *code = h;
  if (h) {
    set_error("device bounds check failed, code " + std::to_string(h));
    return GPW_EDEVICE;
  }
  return GPW_OK;
}

int gpw_profile(gpw_plan_t plan, int enable) {
  if (gpw::bad(plan)) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  if (enable) {
    for (int i = 0; i < GPW_NPHASES; ++i) {
      P.prof_ms[i] = 0.0;
      P.prof_n[i] = 0;
    }
    P.ev_used = 0;
    P.ev_phase.clear();
  }
  P.prof = enable != 0;
  return GPW_OK;
}

int gpw_profile_read(gpw_plan_t plan, double* ms, long long* count, int nphases,
                     long long* launches) {
  if (gpw::bad(plan)) return GPW_EINVAL;
  gpw::Plan& P = plan->p;
  for (size_t i = 0; i < P.ev_phase.size(); ++i) {
    cudaEvent_t a = P.ev_pool[2 * i], b = P.ev_pool[2 * i + 1];
    float t = 0.f;
    cudaError_t e = cudaEventSynchronize(b);
    if (e == cudaSuccess) e = cudaEventElapsedTime(&t, a, b);
    if (e != cudaSuccess) {
      set_error(std::string("gpw_profile_read: ") + cudaGetErrorString(e));
      return GPW_ECUDA;
    }
    P.prof_ms[P.ev_phase[i]] += t;
    P.prof_n[P.ev_phase[i]] += 1;
  }
  P.ev_used = 0;
  P.ev_phase.clear();
  for (int i = 0; i < nphases && i < GPW_NPHASES; ++i) {
    if (ms) ms[i] = P.prof_ms[i];
    if (count) count[i] = P.prof_n[i];
  }
  if (launches) *launches = P.launches;
  return GPW_OK;
}

void gpw_plan_destroy(gpw_plan_t plan) {
  if (!plan) return;
  gpw::free_plan(&plan->p);
  delete plan;
}

void gpw_plan_destroy_async(gpw_plan_t plan, void* stream) {
  if (!plan) return;
  gpw::free_plan(&plan->p, (cudaStream_t)stream, false);
  delete plan;
}

const char* gpw_strerror(int code) {
  switch (code) {
    case GPW_OK: return "ok";
    case GPW_EINVAL: return "invalid argument";
    case GPW_ENOMEM: return "out of memory";
    case GPW_ECUDA: return "CUDA error";
    case GPW_ECUFFT: return "cuFFT error";
    case GPW_ETIMEDOUT: return "timed out";
    case GPW_EDEVICE: return "device bounds check failed";
    case GPW_ERANGE: return "size beyond a fixed limit";
    default: return "unknown error";
  }
}

const char* gpw_last_error(void) { return gpw::g_err.c_str(); }

}  // extern "C"
