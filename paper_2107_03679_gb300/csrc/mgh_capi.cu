// C ABI of the solver (declared in include/mgh.h): parameter validation, device memory of the
// handle, and the entry points that sequence the kernels of the other translation units.
#include <algorithm>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <new>
#include <string>

#include <cmath>

#include "mgh_engine.h"

// The opaque handle of the C ABI is the engine's Handle.
struct mgh_handle : public mgh::Handle {};
static_assert(MGH_MAX_LEVELS == mgh::kMaxLevels, "level arrays of mgh_params and the engine differ");

namespace mgh {

namespace {
thread_local char g_last_error[512] = "";

int coarse_dim(int n) { return (n - 1) / 2 + 1; }

// Validate parameters; fills the level shapes when `lev` is non-null.
mgh_status validate(const mgh_params* p, int* nx_l = nullptr, int* ny_l = nullptr) {
  if (!p) return MGH_INVALID_ARG;
  if (p->nx_int < 1 || p->ny_int < 1 || p->abl < 0) return MGH_INVALID_ARG;
  if (!(p->h > 0.0) || !(p->k > 0.0) || !(p->beta >= 0.0)) return MGH_INVALID_ARG;
  if (p->levels < 2 || p->levels > kMaxLevels) return MGH_INVALID_ARG;
  if (p->nu1 < 0 || p->nu1 > kMaxSweeps || p->nu2 < 0 || p->nu2 > kMaxSweeps) return MGH_INVALID_ARG;
  if (!(p->omega > 0.0 && p->omega <= 1.0)) return MGH_INVALID_ARG;
  if (p->restart < 1 || p->restart > kMaxRestart || p->maxit < 1 || !(p->tol > 0.0)) return MGH_INVALID_ARG;
  if (p->precision != MGH_PREC_FP64 && p->precision != MGH_PREC_MIXED32 && p->precision != MGH_PREC_MIXED16)
    return MGH_INVALID_ARG;
  if (p->batch_max < 1 || p->batch_max > 65535) return MGH_INVALID_ARG;
  if (p->arnoldi != MGH_ARNOLDI_DF && p->arnoldi != MGH_ARNOLDI_FP64 && p->arnoldi != MGH_ARNOLDI_SSTEP)
    return MGH_INVALID_ARG;
  if (p->precision != MGH_PREC_FP64 && p->arnoldi == MGH_ARNOLDI_DF && p->restart > kMaxRestartDf)
    return MGH_INVALID_ARG;
  if (p->precision != MGH_PREC_FP64 && p->arnoldi == MGH_ARNOLDI_SSTEP && p->restart > kMaxRestartSs &&
      p->krylov == MGH_KRYLOV_FGMRES)
    return MGH_INVALID_ARG;
  if (p->krylov != MGH_KRYLOV_FGMRES && p->krylov != MGH_KRYLOV_BICGSTAB && p->krylov != MGH_KRYLOV_IDRS)
    return MGH_INVALID_ARG;
  if (p->cycle_type < 0 || p->cycle_type > kMaxCycleType) return MGH_INVALID_ARG;
  if (p->nu_per_level != 0 && p->nu_per_level != 1) return MGH_INVALID_ARG;
  if (p->nu_per_level)
    for (int l = 0; l + 1 < p->levels; ++l)
      if (p->nu1_level[l] < 0 || p->nu1_level[l] > kMaxSweeps || p->nu2_level[l] < 0 || p->nu2_level[l] > kMaxSweeps)
        return MGH_INVALID_ARG;
  if (p->krylov == MGH_KRYLOV_BICGSTAB && p->restart < 5) return MGH_INVALID_ARG;
  // IDR(s) keeps r, G_0..G_{s-1}, U_0..U_{s-1}, v and t in the restart + 1 basis slots and its
  // scalars (M_s, f, c, alpha, omega, beta, ||r||^2) in the m (m + 1) Hessenberg words
  if (p->krylov == MGH_KRYLOV_IDRS && (p->idr_s < 1 || p->idr_s > kMaxIdrS || p->restart < 2 * p->idr_s + 2))
    return MGH_INVALID_ARG;
  if (!std::isfinite(p->shift_re) || !std::isfinite(p->shift_im)) return MGH_INVALID_ARG;
  const long long nx = p->nx_int + 2LL * p->abl, ny = p->ny_int + 2LL * p->abl;
  if (p->precision == MGH_PREC_MIXED16) {
    // FP16 storage is built into the s-step FGMRES engine and the level-0 wavefront kernels
    // (lane rings of 8-byte FP16 pairs: even rows; both level-0 stages need a sweep)
    const int n1 = p->nu_per_level ? p->nu1_level[0] : p->nu1, n2 = p->nu_per_level ? p->nu2_level[0] : p->nu2;
    if (p->krylov != MGH_KRYLOV_FGMRES || p->arnoldi != MGH_ARNOLDI_SSTEP || p->restart > kMaxRestartSs ||
        nx % 2 != 0 || n1 < 1 || n2 < 1)
      return MGH_NOT_SUPPORTED;
  }
  if (p->deflate < 0 || p->deflate > kMaxDeflate || (p->deflate > 0 && p->deflate >= p->restart))
    return MGH_INVALID_ARG;
  if (p->deflate > 0 && (p->krylov != MGH_KRYLOV_FGMRES ||
                         (p->precision != MGH_PREC_FP64 &&
                          !(p->precision == MGH_PREC_MIXED32 && p->arnoldi == MGH_ARNOLDI_FP64))))
    return MGH_NOT_SUPPORTED;
  if (nx > (1 << 20) || ny > (1 << 20) || nx * ny > (1LL << 31)) return MGH_INVALID_ARG;
  int cx = (int)nx, cy = (int)ny;
  for (int l = 0; l < p->levels; ++l) {
    if (nx_l) { nx_l[l] = cx; ny_l[l] = cy; }
    if (l + 1 < p->levels) { cx = coarse_dim(cx); cy = coarse_dim(cy); }
  }
  if ((long long)cx * cy > kMaxCoarse) return MGH_INVALID_ARG;
  return MGH_OK;
}

size_t pad256(size_t b) { return (b + 255) & ~size_t(255); }

// Complex words of one right-hand side's deflated-restart data: C m x k, Hh (k+1) x k, R k x k,
// the k Givens cosines (real parts) and sines.
// Strips of at least 48 columns across a row: bounds the strips of every fused post launch.
size_t npart_strips(int nx) { return (size_t)(nx + 47) / 48; }

size_t dr_words(int m, int k) { return (size_t)m * k + (size_t)(k + 1) * k + (size_t)k * k + 2 * (size_t)k; }

// Bytes of every device allocation of a handle, in allocation order.
size_t workspace_bytes(const mgh_params& p) {
  int nxl[kMaxLevels], nyl[kMaxLevels];
  validate(&p, nxl, nyl);
  const size_t B = p.batch_max, m = p.restart;
  const size_t cs = p.precision == MGH_PREC_FP64 ? 16 : 8;
  const size_t N = (size_t)nxl[0] * nyl[0], Np = (N + 63) / 64 * 64;
  size_t t = 0;
  for (int l = 0; l < p.levels; ++l) {
    const size_t n = (size_t)nxl[l] * nyl[l];
    t += pad256(8 * n) + 2 * pad256(cs * n);
    if (l >= 1) t += 2 * pad256(cs * n * B);             // b, vfin
    if (l + 1 < p.levels) t += pad256(cs * n * B);       // vpre
    if (p.cycle_type >= 2 && l >= 1 && l + 1 < p.levels) t += pad256(cs * n * B);   // wacc
  }
  const size_t nc = (size_t)nxl[p.levels - 1] * nyl[p.levels - 1];
  const size_t W = 3 * (size_t)nxl[p.levels - 1] + 1;
  t += pad256(8 * (size_t)p.nx_int * p.ny_int) + pad256(16 * N);
  t += pad256(16 * nc * W) + pad256(4 * nc) + 2 * pad256(16 * nc * nc) + pad256(8 * nc * nc) + pad256(4);
  t += pad256(16 * B * (m + 1) * Np) + pad256(cs * B * m * N) + pad256(16 * B * Np) + 2 * pad256(16 * B * N);
  t += pad256(16 * B * m * (m + 1)) + 2 * pad256(16 * B * (m + 1)) + pad256(8 * B * m) + pad256(16 * B * m);
  t += pad256(16 * B * (m + 1)) + pad256(16 * B * m) + pad256(8 * B * (m + 1)) + pad256(sizeof(RhsState) * B);
  t += pad256(16 * (1216 + B) * partial_stride(m)) + pad256(8 * (B + 1));
  t += pad256(16 * Np) + pad256(16 * B * (m + 1)) + pad256(16 * B * 2 * m) + pad256(4);   // DAdf, hpend, coef, err
  t += pad256(56 * (size_t)p.nx_int * p.ny_int);                                          // tvbuf
  if (p.precision != MGH_PREC_FP64) t += 2 * pad256(16 * B * Np);                        // xdf, bdf
  if (p.precision != MGH_PREC_FP64) t += pad256(4 * B * (size_t)nyl[0] * npart_strips(nxl[0]));   // npart
  if (p.deflate > 0)                                                                       // Hraw, drbuf, dr_mode
    t += pad256(16 * B * m * (m + 1)) + pad256(16 * B * dr_words(p.restart, p.deflate)) + pad256(4 * B) +
         pad256(16 * B * (m + 1));
  return t;
}

template <typename T>
mgh_status dev_alloc(T** p, size_t bytes) {
  cudaError_t e = cudaMalloc((void**)p, std::max<size_t>(bytes, 1));
  if (e != cudaSuccess) {
    set_error("cudaMalloc", e, __FILE__, __LINE__);
    *p = nullptr;
    return e == cudaErrorMemoryAllocation ? MGH_OUT_OF_MEMORY : MGH_CUDA_ERROR;
  }
  return MGH_OK;
}

void free_handle(mgh_handle* h) {
  if (!h) return;
  for (int l = 0; l < kMaxLevels; ++l) {
    Level& lv = h->lev[l];
    cudaFree(lv.c); cudaFree(lv.D); cudaFree(lv.wDinv); cudaFree(lv.b); cudaFree(lv.vpre); cudaFree(lv.vfin);
    cudaFree(lv.wacc);
  }
  cudaFree(h->f_d); cudaFree(h->DA); cudaFree(h->band); cudaFree(h->piv); cudaFree(h->kinv64); cudaFree(h->kinv64r);
  cudaFree(h->kinv32); cudaFree(h->lu_info); cudaFree(h->V); cudaFree(h->Z); cudaFree(h->W);
  cudaFree(h->T1); cudaFree(h->T2); cudaFree(h->H); cudaFree(h->hcol); cudaFree(h->h2col); cudaFree(h->cs);
  cudaFree(h->sn); cudaFree(h->g); cudaFree(h->y); cudaFree(h->vscale); cudaFree(h->st); cudaFree(h->partial);
  cudaFree(h->hs_f); cudaFree(h->hs_theta); cudaFree(h->hs_u); cudaFree(h->hs_G); cudaFree(h->hs_rec);
  cudaFree(h->hs_y); cudaFree(h->hs_r);
  cudaFree(h->dscratch); cudaFree(h->DAdf); cudaFree(h->hpend); cudaFree(h->coef);
  cudaFree(h->dev_err); cudaFree(h->xdf); cudaFree(h->bdf); cudaFree(h->tvbuf);
  cudaFree(h->Hraw); cudaFree(h->drbuf); cudaFree(h->dr_mode); cudaFree(h->g0); cudaFree(h->npart);
  if (h->st_host) cudaFreeHost(h->st_host);
  if (h->dr_hraw_host) cudaFreeHost(h->dr_hraw_host);
  if (h->dr_host) cudaFreeHost(h->dr_host);
  if (h->dr_mode_host) cudaFreeHost(h->dr_mode_host);
  if (h->dr_g0_host) cudaFreeHost(h->dr_g0_host);
  if (h->dr_y_host) cudaFreeHost(h->dr_y_host);
  for (cudaEvent_t e : h->ev) cudaEventDestroy(e);
  if (h->gev_in) cudaEventDestroy(h->gev_in);
  if (h->gev_out) cudaEventDestroy(h->gev_out);
  if (h->gstream) cudaStreamDestroy(h->gstream);
  delete[] h->tma;
  delete[] h->tma_in;
  delete h;
}

// The handle exists and its device is the current one (kernels and streams belong to it).
bool handle_ok(const Handle* h) {
  if (!h) return false;
  int dev = -1;
  return cudaGetDevice(&dev) == cudaSuccess && dev == h->device;
}

bool batch_ok(const Handle* h, int B) { return handle_ok(h) && B >= 1 && B <= h->Bmax; }

}  // namespace

ProfScope::ProfScope(Handle& hh, int cls) : h(hh) {
  if (!h.prof) return;
  if (h.ev_used + 2 > h.ev.size()) {
    const size_t grow = std::max<size_t>(256, h.ev.size());
    for (size_t i = 0; i < grow; ++i) {
      cudaEvent_t e;
      if (cudaEventCreate(&e) != cudaSuccess) return;   // profiling degrades, the launch still runs
      h.ev.push_back(e);
    }
  }
  slot = (int)h.ev_used;
  h.ev_used += 2;
  if (h.ev_cls.size() < h.ev_used / 2) h.ev_cls.resize(h.ev_used / 2);
  h.ev_cls[slot / 2] = cls;
  cudaEventRecord(h.ev[slot], h.stream);
}

ProfScope::~ProfScope() {
  if (slot >= 0) cudaEventRecord(h.ev[slot + 1], h.stream);
}

mgh_status prof_flush(Handle& h) {
  for (size_t i = 0; i + 1 < h.ev_used; i += 2) {
    float ms = 0.f;
    MGH_CUDA(cudaEventElapsedTime(&ms, h.ev[i], h.ev[i + 1]));
    const int c = h.ev_cls[i / 2];
    h.acc.ms[c] += ms;
    h.acc.launches[c] += 1;
  }
  h.ev_used = 0;
  return MGH_OK;
}

void set_error(const char* what, cudaError_t e, const char* file, int line) {
  std::snprintf(g_last_error, sizeof(g_last_error), "%s failed: %s (%s:%d)", what, cudaGetErrorString(e), file,
                line);
}

}  // namespace mgh

using namespace mgh;

extern "C" {

void mgh_default_params(mgh_params* p) {
  if (!p) return;
  std::memset(p, 0, sizeof(*p));
  p->nx_int = 128; p->ny_int = 128; p->abl = 16;
  p->h = 1.0; p->k = 2.0 * 3.14159265358979323846 / 10.0; p->beta = 0.15;
  p->shift_re = 1.0; p->shift_im = 0.5;
  p->levels = 4; p->nu1 = 2; p->nu2 = 2; p->omega = 0.8;
  p->restart = 20; p->maxit = 5000; p->tol = 1e-8;
  p->precision = MGH_PREC_FP64; p->batch_max = 1;
  p->idr_s = 4;
}

mgh_status mgh_workspace_bytes(const mgh_params* p, size_t* bytes) {
  if (!bytes) return MGH_INVALID_ARG;
  MGH_TRY(validate(p));
  *bytes = workspace_bytes(*p);
  return MGH_OK;
}

mgh_status mgh_create(const mgh_params* p, void* cuda_stream, mgh_handle** out) {
  if (!out) return MGH_INVALID_ARG;
  *out = nullptr;
  int nxl[kMaxLevels], nyl[kMaxLevels];
  MGH_TRY(validate(p, nxl, nyl));
  mgh_handle* h = new (std::nothrow) mgh_handle();
  if (!h) return MGH_OUT_OF_MEMORY;
  h->p = *p;
  h->stream = (cudaStream_t)cuda_stream;
  {
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) { set_error("cudaGetDevice", e, __FILE__, __LINE__); delete h; return MGH_CUDA_ERROR; }
    h->device = dev;
    cudaDeviceGetAttribute(&h->num_sms, cudaDevAttrMultiProcessorCount, dev);
    if (h->num_sms < 1) h->num_sms = 1;
  }
  h->nx = nxl[0]; h->ny = nyl[0]; h->N = (size_t)h->nx * h->ny;
  h->Np = (h->N + 63) / 64 * 64;
  h->L = p->levels;
  h->fp64 = p->precision == MGH_PREC_FP64;
  h->half = p->precision == MGH_PREC_MIXED16;
  if (h->half) {   // scale sqrt(N)/16 rounded to a power of two: FP16 values near 1/16 in RMS
    const double t = std::sqrt((double)nxl[0] * nyl[0]) / 16.0;
    h->zmul = (float)std::ldexp(1.0, std::max(0, (int)std::lround(std::log2(std::max(t, 1.0)))));
  }
  h->csize = h->fp64 ? 16 : 8;
  h->m = p->restart;
  h->Bmax = p->batch_max;
  const size_t B = h->Bmax, m = h->m, N = h->N, Np = h->Np, cs = h->csize;
  mgh_status s = MGH_OK;
#define ALLOC(ptr, bytes) do { s = dev_alloc(&(ptr), (bytes)); if (s != MGH_OK) { free_handle(h); return s; } } while (0)
  double hl = p->h;
  int sc = 1;
  for (int l = 0; l < h->L; ++l) {
    Level& lv = h->lev[l];
    lv.nx = nxl[l]; lv.ny = nyl[l]; lv.h = hl; lv.scale = sc;
    const size_t n = lv.n();
    ALLOC(lv.c, 8 * n);
    ALLOC(lv.D, cs * n);
    ALLOC(lv.wDinv, cs * n);
    if (l >= 1) { ALLOC(lv.b, cs * n * B); ALLOC(lv.vfin, cs * n * B); }
    if (l + 1 < h->L) ALLOC(lv.vpre, cs * n * B);
    if (p->cycle_type >= 2 && l >= 1 && l + 1 < h->L) ALLOC(lv.wacc, cs * n * B);
    hl *= 2.0; sc *= 2;
  }
  const Level& cl = h->lev[h->L - 1];
  h->nc = (int)cl.n();
  const size_t nc = h->nc, W = 3 * (size_t)cl.nx + 1;
  ALLOC(h->f_d, 8 * (size_t)p->nx_int * p->ny_int);
  ALLOC(h->DA, 16 * N);
  ALLOC(h->band, 16 * nc * W);
  ALLOC(h->piv, 4 * nc);
  ALLOC(h->kinv64, 16 * nc * nc);
  ALLOC(h->kinv64r, 16 * nc * nc);
  if (!h->fp64) ALLOC(h->kinv32, 8 * nc * nc);
  ALLOC(h->lu_info, 4);
  ALLOC(h->V, 16 * B * (m + 1) * Np);
  ALLOC(h->Z, cs * B * m * N);
  ALLOC(h->W, 16 * B * Np);
  ALLOC(h->T1, 16 * B * N);
  ALLOC(h->T2, 16 * B * N);
  ALLOC(h->H, 16 * B * m * (m + 1));
  ALLOC(h->hcol, 16 * B * (m + 1));
  ALLOC(h->h2col, 16 * B * (m + 1));
  ALLOC(h->cs, 8 * B * m);
  ALLOC(h->sn, 16 * B * m);
  ALLOC(h->g, 16 * B * (m + 1));
  ALLOC(h->y, 16 * B * m);
  ALLOC(h->vscale, 8 * B * (m + 1));
  ALLOC(h->st, sizeof(RhsState) * B);
  ALLOC(h->partial, 16 * (1216 + B) * partial_stride(m));
  ALLOC(h->DAdf, 16 * Np);
  ALLOC(h->dev_err, 4);
  if (!h->fp64) { ALLOC(h->xdf, 16 * B * Np); ALLOC(h->bdf, 16 * B * Np); }
  ALLOC(h->hpend, 16 * B * (m + 1));
  ALLOC(h->coef, 16 * B * 2 * m);
  ALLOC(h->dscratch, 8 * (B + 1));
  ALLOC(h->tvbuf, 56 * (size_t)p->nx_int * p->ny_int);
  if (!h->fp64) ALLOC(h->npart, 4 * B * (size_t)h->ny * npart_strips(h->nx));
  if (p->deflate > 0) {
    ALLOC(h->Hraw, 16 * B * m * (m + 1));
    ALLOC(h->drbuf, 16 * B * dr_words(p->restart, p->deflate));
    ALLOC(h->dr_mode, 4 * B);
    ALLOC(h->g0, 16 * B * (m + 1));
  }
#undef ALLOC
  if (cudaMallocHost((void**)&h->st_host, sizeof(RhsState) * B) != cudaSuccess) {
    h->st_host = nullptr;
    free_handle(h);
    return MGH_OUT_OF_MEMORY;
  }
  if (p->deflate > 0) {
    bool ok = true;
    if (cudaMallocHost((void**)&h->dr_hraw_host, 16 * B * m * (m + 1)) != cudaSuccess) { h->dr_hraw_host = nullptr; ok = false; }
    if (ok && cudaMallocHost((void**)&h->dr_host, 16 * B * dr_words(p->restart, p->deflate)) != cudaSuccess) {
      h->dr_host = nullptr;
      ok = false;
    }
    if (ok && cudaMallocHost((void**)&h->dr_mode_host, 4 * B) != cudaSuccess) { h->dr_mode_host = nullptr; ok = false; }
    if (ok && cudaMallocHost((void**)&h->dr_g0_host, 16 * B * (m + 1)) != cudaSuccess) { h->dr_g0_host = nullptr; ok = false; }
    if (ok && cudaMallocHost((void**)&h->dr_y_host, 16 * B * m) != cudaSuccess) { h->dr_y_host = nullptr; ok = false; }
    if (!ok) { free_handle(h); return MGH_OUT_OF_MEMORY; }
  }
  // level-kernel selection (environment): MGH_VCYCLE=tile picks the shared-memory tile kernels
  // for the FP32 levels; MGH_WAVE_SEG sets the rows per warp of the wavefront kernels,
  // MGH_WAVE_MIN_NX the narrowest level that uses them, MGH_WAVE_PF their load depth in rows,
  // MGH_WAVE_WARPS their warps per block and MGH_WAVE_RING the length of their shared-memory row
  // rings in unroll periods (0: loads prefetched into registers); MGH_WAVE_FILL=bulk fills the
  // rings with bulk copies issued by one lane instead of per-lane cp.async copies
  if (const char* e = std::getenv("MGH_VCYCLE")) h->vc_wave = std::strcmp(e, "tile") != 0;
  if (const char* e = std::getenv("MGH_WAVE_SEG")) h->wave_seg = std::max(0, std::atoi(e));
  if (const char* e = std::getenv("MGH_WAVE_MIN_NX")) h->wave_min_nx = std::max(0, std::atoi(e));
  if (const char* e = std::getenv("MGH_WAVE_PF")) h->wave_pf = std::atoi(e) == 2 ? 2 : 1;
  if (const char* e = std::getenv("MGH_WAVE_WARPS")) h->wave_warps = std::atoi(e) == 2 ? 2 : 4;
  if (const char* e = std::getenv("MGH_WAVE_RING")) h->wave_ring = std::max(0, std::atoi(e));
  if (const char* e = std::getenv("MGH_WAVE_FILL")) h->wave_lane_ring = std::strcmp(e, "bulk") != 0;
  if (h->half) {   // the FP16 level-0 kernels exist only as lane-ring wavefront kernels
    h->vc_wave = true;
    h->wave_min_nx = 0;
    h->wave_ring = 1;
    h->wave_lane_ring = true;
  }
  // MGH_GRAPHS=0 issues every restart cycle's launches directly instead of replaying a CUDA graph
  if (const char* e = std::getenv("MGH_GRAPHS")) h->use_graphs = std::strcmp(e, "0") != 0;
  // the coarse levels whose fields fit in one block's shared memory run as one kernel per cycle;
  // MGH_TAIL=0 keeps every level on the level kernels
  h->tail_l0 = choose_tail_level(*h);
  if (const char* e = std::getenv("MGH_TAIL")) if (std::strcmp(e, "0") == 0) h->tail_l0 = 0;
  // MGH_DEFLATE_FORCE_PLAIN=1 sends every deflated restart down its plain-restart fallback (tests)
  if (const char* e = std::getenv("MGH_DEFLATE_FORCE_PLAIN")) if (std::strcmp(e, "1") == 0) h->dr_force_plain = true;
  // MGH_GRAM8=0 sums the s-step Gram matrix with four groups of 64 threads (two blocks per SM)
  // instead of eight one-warp groups (three blocks per SM)
  if (const char* e = std::getenv("MGH_GRAM8")) if (std::strcmp(e, "0") == 0) h->gram8 = false;
  // MGH_FUSE_MATVEC=0 keeps the s-step operator product in its own kernel
  if (const char* e = std::getenv("MGH_FUSE_MATVEC")) if (std::strcmp(e, "0") == 0) h->fuse_ok = false;
  // MGH_TAIL_CLUSTER=2|4 runs the tail over a cluster of that many blocks per right-hand side
  if (const char* e = std::getenv("MGH_TAIL_CLUSTER")) {
    const int c = std::atoi(e);
    if (h->tail_l0 > 0 && tail_cluster_fits(*h, h->tail_l0, c)) h->tail_cluster = c;
  }
  s = build_vcycle_tma(*h);
  if (s != MGH_OK) { free_handle(h); return s; }
  // start from f_d = 0 so that every later call finds a complete operator
  cudaError_t e = cudaMemsetAsync(h->T1, 0, 8 * (size_t)p->nx_int * p->ny_int, h->stream);
  if (e != cudaSuccess) { set_error("cudaMemsetAsync", e, __FILE__, __LINE__); free_handle(h); return MGH_CUDA_ERROR; }
  s = setup_contrast(*h, (const double*)h->T1);
  if (s != MGH_OK) { free_handle(h); return s; }
  *out = h;
  return MGH_OK;
}

void mgh_destroy(mgh_handle* h) {
  if (!h) return;
  cudaStreamSynchronize(h->stream);
  free_handle(h);
}

mgh_status mgh_set_contrast(mgh_handle* h, const double* f_d) {
  if (!handle_ok(h) || !f_d) return MGH_INVALID_ARG;
  return setup_contrast(*h, f_d);
}

mgh_status mgh_incident_field(mgh_handle* h, const double* theta, int B, mgh_cdouble* u_in) {
  if (!batch_ok(h, B) || !theta || !u_in) return MGH_INVALID_ARG;
  return launch_incident(*h, theta, B, (cd*)u_in, false);
}

mgh_status mgh_rhs(mgh_handle* h, const double* theta, int B, mgh_cdouble* b) {
  if (!batch_ok(h, B) || !theta || !b) return MGH_INVALID_ARG;
  return launch_incident(*h, theta, B, (cd*)b, true);
}

mgh_status mgh_apply(mgh_handle* h, const mgh_cdouble* x, int B, mgh_cdouble* y) {
  if (!batch_ok(h, B) || !x || !y || x == y) return MGH_INVALID_ARG;
  return launch_apply_A(*h, (const cd*)x, B, (cd*)y);
}

mgh_status mgh_precondition(mgh_handle* h, const mgh_cdouble* b, int B, mgh_cdouble* z) {
  if (!batch_ok(h, B) || !b || !z || (const void*)b == (const void*)z) return MGH_INVALID_ARG;
  return vcycle(*h, (const cd*)b, h->N, nullptr, 0, z, h->N, true, B, nullptr);
}

mgh_status mgh_coarse_solve(mgh_handle* h, const mgh_cdouble* b, int B, mgh_cdouble* x) {
  if (!batch_ok(h, B) || !b || !x || (const void*)b == (const void*)x) return MGH_INVALID_ARG;
  return launch_coarse_apply(*h, b, (size_t)h->nc, x, (size_t)h->nc, B, nullptr, true);
}

mgh_status mgh_level_shape(const mgh_handle* h, int level, int* nx, int* ny, double* h_level) {
  if (!h || level < 0 || level >= h->L) return MGH_INVALID_ARG;
  if (nx) *nx = h->lev[level].nx;
  if (ny) *ny = h->lev[level].ny;
  if (h_level) *h_level = h->lev[level].h;
  return MGH_OK;
}

mgh_status mgh_level_coefficient(mgh_handle* h, int level, double* c) {
  if (!handle_ok(h) || !c || level < 0 || level >= h->L) return MGH_INVALID_ARG;
  MGH_CUDA(cudaMemcpyAsync(c, h->lev[level].c, 8 * h->lev[level].n(), cudaMemcpyDeviceToDevice, h->stream));
  return MGH_OK;
}

mgh_status mgh_solve(mgh_handle* h, const mgh_cdouble* b, int B, mgh_cdouble* x, mgh_solve_info* info) {
  if (!batch_ok(h, B) || !b || !x || (const void*)b == (const void*)x) return MGH_INVALID_ARG;
  return fgmres_solve(*h, (const cd*)b, B, (cd*)x, info);
}

mgh_status mgh_forward(mgh_handle* h, const double* theta, int B, mgh_cdouble* u_sc, mgh_solve_info* info) {
  if (!batch_ok(h, B) || !theta || !u_sc) return MGH_INVALID_ARG;
  MGH_TRY(launch_incident(*h, theta, B, h->T1, true));
  MGH_CUDA(cudaMemsetAsync(u_sc, 0, 16 * h->N * B, h->stream));
  return fgmres_solve(*h, h->T1, B, (cd*)u_sc, info);
}

mgh_status mgh_crop(mgh_handle* h, const mgh_cdouble* u, int B, mgh_cdouble* u_int) {
  if (!batch_ok(h, B) || !u || !u_int) return MGH_INVALID_ARG;
  return launch_crop(*h, (const cd*)u, B, (cd*)u_int);
}

mgh_status mgh_sample(mgh_handle* h, const mgh_cdouble* u, int B, const int64_t* rec, int M, mgh_cdouble* out) {
  if (!batch_ok(h, B) || !u || !rec || !out || M < 1) return MGH_INVALID_ARG;
  return launch_sample(*h, (const cd*)u, B, rec, M, (cd*)out);
}

mgh_status mgh_scatter(mgh_handle* h, const mgh_cdouble* vals, int B, const int64_t* rec, int M, mgh_cdouble* G) {
  if (!batch_ok(h, B) || !vals || !rec || !G || M < 1) return MGH_INVALID_ARG;
  return launch_scatter(*h, (const cd*)vals, B, rec, M, (cd*)G);
}

mgh_status mgh_misfit(mgh_handle* h, const mgh_cdouble* u, const mgh_cdouble* y, int B, const int64_t* rec, int M,
                      mgh_cdouble* r, mgh_cdouble* G, double* loss_host) {
  if (!batch_ok(h, B) || !u || !y || !rec || M < 1) return MGH_INVALID_ARG;
  MGH_TRY(launch_misfit(*h, (const cd*)u, (const cd*)y, B, rec, M, (cd*)r, (cd*)G, h->dscratch + B));
  if (loss_host) {
    MGH_CUDA(cudaMemcpyAsync(loss_host, h->dscratch + B, 8, cudaMemcpyDeviceToHost, h->stream));
    MGH_CUDA(cudaStreamSynchronize(h->stream));
  }
  return MGH_OK;
}

mgh_status mgh_gradient(mgh_handle* h, const double* theta, const mgh_cdouble* u_sc, const mgh_cdouble* G, int B,
                        double* grad, mgh_solve_info* info) {
  if (!batch_ok(h, B) || !theta || !u_sc || !G || !grad) return MGH_INVALID_ARG;
  MGH_TRY(launch_conj(*h, (const cd*)G, B, h->T1));
  MGH_CUDA(cudaMemsetAsync(h->T2, 0, 16 * h->N * B, h->stream));
  const mgh_status s = fgmres_solve(*h, h->T1, B, h->T2, info);
  if (s != MGH_OK && s != MGH_NOT_CONVERGED) return s;
  MGH_TRY(launch_gradient(*h, theta, (const cd*)u_sc, h->T2, B, grad));
  return s;
}

mgh_status mgh_data_term_gradient_host(mgh_handle* h, const double* f_d, const double* theta, int B,
                                       const int64_t* rec, int M, const mgh_cdouble* y, double* grad, double* loss,
                                       mgh_cdouble* r, mgh_solve_info* info_fwd, mgh_solve_info* info_adj) {
  if (!batch_ok(h, B) || !f_d || !theta || !rec || !y || !grad || !loss || M < 1) return MGH_INVALID_ARG;
  const size_t Bm = h->Bmax, N = h->N, nint = (size_t)h->p.nx_int * h->p.ny_int;
  cudaStream_t s = h->stream;
  // device staging, allocated once per handle (the receiver buffers again when M grows)
  if (!h->hs_f) {
    MGH_TRY(dev_alloc(&h->hs_f, 8 * nint));
    MGH_TRY(dev_alloc(&h->hs_theta, 8 * Bm));
    MGH_TRY(dev_alloc(&h->hs_u, 16 * Bm * N));
    MGH_TRY(dev_alloc(&h->hs_G, 16 * Bm * N));
  }
  if (M > h->hs_M) {
    MGH_CUDA(cudaStreamSynchronize(s));
    cudaFree(h->hs_rec); cudaFree(h->hs_y); cudaFree(h->hs_r);
    h->hs_rec = nullptr; h->hs_y = nullptr; h->hs_r = nullptr; h->hs_M = 0;
    MGH_TRY(dev_alloc(&h->hs_rec, 8 * (size_t)M));
    MGH_TRY(dev_alloc(&h->hs_y, 16 * Bm * M));
    MGH_TRY(dev_alloc(&h->hs_r, 16 * Bm * M));
    h->hs_M = M;
  }
  // inputs in
  MGH_CUDA(cudaMemcpyAsync(h->hs_f, f_d, 8 * nint, cudaMemcpyHostToDevice, s));
  MGH_CUDA(cudaMemcpyAsync(h->hs_theta, theta, 8 * (size_t)B, cudaMemcpyHostToDevice, s));
  MGH_CUDA(cudaMemcpyAsync(h->hs_rec, rec, 8 * (size_t)M, cudaMemcpyHostToDevice, s));
  MGH_CUDA(cudaMemcpyAsync(h->hs_y, y, 16 * (size_t)B * M, cudaMemcpyHostToDevice, s));
  // contrast, forward solves, misfit, adjoint solves and gradient: the device-pointer path
  MGH_TRY(setup_contrast(*h, h->hs_f));
  MGH_TRY(launch_incident(*h, h->hs_theta, B, h->T1, true));
  MGH_CUDA(cudaMemsetAsync(h->hs_u, 0, 16 * N * B, s));
  const mgh_status sf = fgmres_solve(*h, h->T1, B, h->hs_u, info_fwd);
  if (sf != MGH_OK && sf != MGH_NOT_CONVERGED) return sf;
  MGH_TRY(launch_misfit(*h, h->hs_u, h->hs_y, B, h->hs_rec, M, h->hs_r, h->hs_G, h->dscratch + B));
  MGH_TRY(launch_conj(*h, h->hs_G, B, h->T1));
  MGH_CUDA(cudaMemsetAsync(h->T2, 0, 16 * N * B, s));
  const mgh_status sa = fgmres_solve(*h, h->T1, B, h->T2, info_adj);
  if (sa != MGH_OK && sa != MGH_NOT_CONVERGED) return sa;
  MGH_TRY(launch_gradient(*h, h->hs_theta, h->hs_u, h->T2, B, h->hs_f));
  // results out
  MGH_CUDA(cudaMemcpyAsync(grad, h->hs_f, 8 * nint, cudaMemcpyDeviceToHost, s));
  MGH_CUDA(cudaMemcpyAsync(loss, h->dscratch + B, 8, cudaMemcpyDeviceToHost, s));
  if (r) MGH_CUDA(cudaMemcpyAsync(r, h->hs_r, 16 * (size_t)B * M, cudaMemcpyDeviceToHost, s));
  MGH_CUDA(cudaStreamSynchronize(s));
  return sf != MGH_OK ? sf : sa;
}

mgh_status mgh_tv_prox(mgh_handle* h, const double* fbar, const double* d, double gamma, double lam,
                       int iters, double* out) {
  if (!handle_ok(h) || !fbar || !out || iters < 1 || !(lam >= 0.0) || !std::isfinite(lam) || !std::isfinite(gamma))
    return MGH_INVALID_ARG;
  return tv_prox(*h, fbar, d, gamma, lam, iters, out);
}

mgh_status mgh_fbs_momentum(mgh_handle* h, const double* f, const double* f_prev, double c, double* fbar) {
  if (!handle_ok(h) || !f || !f_prev || !fbar || !std::isfinite(c)) return MGH_INVALID_ARG;
  return fbs_momentum(*h, f, f_prev, c, fbar);
}

mgh_status mgh_profile_enable(mgh_handle* h, int enable) {
  if (!handle_ok(h)) return MGH_INVALID_ARG;
  MGH_CUDA(cudaStreamSynchronize(h->stream));
  MGH_TRY(prof_flush(*h));
  h->acc = mgh_profile{};
  h->prof = enable != 0;
  return MGH_OK;
}

mgh_status mgh_profile_read(mgh_handle* h, mgh_profile* out) {
  if (!handle_ok(h) || !out) return MGH_INVALID_ARG;
  MGH_CUDA(cudaStreamSynchronize(h->stream));
  MGH_TRY(prof_flush(*h));
  *out = h->acc;
  return MGH_OK;
}

mgh_status mgh_get_kernel_shape(const mgh_handle* h, mgh_kernel_shape* out) {
  if (!h || !out) return MGH_INVALID_ARG;
  for (int l = 0; l < kMaxLevels; ++l) out->wave_seg[l] = h->wave_seg_level[l];
  out->wave_warps = h->wave_warps;
  out->wave_ring = h->wave_ring;
  out->tail_level = h->tail_l0;
  out->tail_cluster = h->tail_cluster;
  return MGH_OK;
}

mgh_status mgh_set_kernel_shape(mgh_handle* h, const mgh_kernel_shape* s) {
  if (!handle_ok(h) || !s) return MGH_INVALID_ARG;
  for (int l = 0; l < kMaxLevels; ++l)
    if (s->wave_seg[l] < 0 || s->wave_seg[l] > 4096) return MGH_INVALID_ARG;
  if (s->wave_warps != 2 && s->wave_warps != 4) return MGH_INVALID_ARG;
  if (s->wave_ring != 1 && s->wave_ring != 2) return MGH_INVALID_ARG;
  if (s->tail_level < -1 || s->tail_level > h->L - 2) return MGH_INVALID_ARG;
  if (s->tail_level > 0 && !tail_level_fits(*h, s->tail_level)) return MGH_INVALID_ARG;
  if (s->tail_cluster != 0 && s->tail_cluster != 1 && s->tail_cluster != 2 && s->tail_cluster != 4)
    return MGH_INVALID_ARG;
  const int l0 = s->tail_level < 0 ? choose_tail_level(*h) : s->tail_level;
  const int cl = s->tail_cluster;
  if (cl > 1 && (l0 == 0 || !tail_cluster_fits(*h, l0, cl))) return MGH_INVALID_ARG;
  if (h->half && (s->wave_warps != 4 || s->wave_ring != 1)) return MGH_NOT_SUPPORTED;
  MGH_CUDA(cudaStreamSynchronize(h->stream));   // launches already queued keep their shapes
  for (int l = 0; l < kMaxLevels; ++l) h->wave_seg_level[l] = s->wave_seg[l];
  h->wave_warps = s->wave_warps;
  h->wave_ring = s->wave_ring;
  h->tail_l0 = l0;
  h->tail_cluster = cl;
  return MGH_OK;
}

mgh_status mgh_debug_inject_timeout(mgh_handle* h) {
  if (!handle_ok(h)) return MGH_INVALID_ARG;
  if (h->fp64 || h->p.krylov != MGH_KRYLOV_FGMRES || h->p.arnoldi == MGH_ARNOLDI_FP64) return MGH_NOT_SUPPORTED;
  h->inject_timeout = true;
  return MGH_OK;
}

uint64_t mgh_launch_count(const mgh_handle* h, int reset) {
  if (!h) return 0;
  const uint64_t n = h->launches;
  if (reset) const_cast<mgh_handle*>(h)->launches = 0;
  return n;
}

const char* mgh_status_string(mgh_status s) {
  switch (s) {
    case MGH_OK: return "ok";
    case MGH_INVALID_ARG: return "invalid argument";
    case MGH_NOT_CONVERGED: return "not converged";
    case MGH_CUDA_ERROR: return "CUDA error";
    case MGH_OUT_OF_MEMORY: return "out of device memory";
    case MGH_TIMEOUT: return "device wait timed out";
    case MGH_NOT_SUPPORTED: return "not supported";
  }
  return "unknown status";
}

const char* mgh_last_error(void) { return mgh::g_last_error; }

}  // extern "C"
