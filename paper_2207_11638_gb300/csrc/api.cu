// C ABI (include/cdct.h): argument checking, plans and kernel dispatch.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>
#include <atomic>
#include <cstring>
#include <mutex>
#include <algorithm>
#include <new>
#include <string>
#include <vector>

#include "../../include/cdct.h"
#include "butterfly.cuh"
#include "cnn.cuh"
#include "common.cuh"

using namespace cdct;

// Device word the kernels set when a bounded wait gives up (see
// cdct_check_device); one per device, reached through its symbol address.
static __device__ int g_device_error;

// Scratch of cdct_fwd_zonal_inv_noalloc: room for the per-CTA / per-warp
// error partials of one call.  Device code reaches it through the address
// the host fetches once per device (host code must not use the symbol
// itself: in host code it names a host-side stand-in, not device memory).
constexpr size_t kNoAllocScratchDoubles = size_t(1) << 17;   // 1 MiB
static __device__ __align__(256) double g_noalloc_scratch[kNoAllocScratchDoubles];

struct cdct_batch_s;

// Failure-detection test hook (cdct_set_fault_injection).
static std::atomic<int> g_fault_mode{0};
static std::atomic<long long> g_fault_limit{kDefaultWaitLimit};

namespace cdct {
int fault_mode(long long* wait_limit) {
  const int m = g_fault_mode.load();
  if (wait_limit != nullptr) *wait_limit = m ? g_fault_limit.load() : kDefaultWaitLimit;
  return m;
}
}  // namespace cdct

struct cdct_rd_s {
  int variant;
  int tables[3 * 32 + 32 * 32 + 16 * 16 + 8 * 8];   // host copy, passed to each launch by value
};

struct cdct_plan_s {
  int n, variant, conv;
  PipeTuning tuning;
  double T[32 * 32];
  double U[32 * 32];
  double S[32];
  float s_f[32];
  KernelSet ks[2];  // per input dtype
};

struct cdct_batch_s {
  const cdct_plan_s* plan;
  int dtype, n_images;
  long long total_units;
  long long total_pixels;
  size_t table_bytes, prefix_offset, map_offset;
  std::string host_table;        // BatchImage[n], int64 unit_prefix[n + 1], UnitDesc[units] (16-byte aligned)
};

namespace {

thread_local std::string g_err;

cdct_status fail(cdct_status st, const std::string& msg) {
  g_err = msg;
  return st;
}

cdct_status cuda_fail(int code, const char* where) {
  return fail(CDCT_ECUDA, std::string(where) + ": " + cudaGetErrorString(static_cast<cudaError_t>(code)));
}

constexpr int rows_per_thread(int n) { return 64 / n; }
constexpr int threads_per_block(int n) { return n / rows_per_thread(n); }
constexpr int blocks_per_cta(int n) { return kThreads / threads_per_block(n); }

bool aligned16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

constexpr int kMaxDevices = 64;

// per-device cache of the SM count and of the error word's address; the
// first call on a device fills it under g_dev_mutex, later calls read it
// after seeing `ready` (so first calls from several threads do not race)
struct DeviceInfo {
  int sms = 0;
  int* err = nullptr;
  double* noalloc_scratch = nullptr;   // device address of g_noalloc_scratch
  std::atomic<bool> ready{false};
  std::atomic<bool> scratch_ready{false};
};
DeviceInfo g_dev[kMaxDevices];
std::mutex g_dev_mutex;

int device_info(DeviceInfo** out) {
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return static_cast<int>(e);
  if (dev < 0 || dev >= kMaxDevices) return static_cast<int>(cudaErrorInvalidDevice);
  DeviceInfo& d = g_dev[dev];
  if (!d.ready.load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if (!d.ready.load(std::memory_order_relaxed)) {
      int sms = 0;
      e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
      if (e != cudaSuccess) return static_cast<int>(e);
      void* p = nullptr;
      e = cudaGetSymbolAddress(&p, g_device_error);
      if (e != cudaSuccess) return static_cast<int>(e);
      d.sms = sms;
      d.err = static_cast<int*>(p);
      d.ready.store(true, std::memory_order_release);
    }
  }
  *out = &d;
  return 0;
}

int pipe_launch(int n, int variant, int conv, int dtype, const PipeArgs& pa, int r, int sms, PipeTuning t,
                void* stream) {
  if (n == 8) return pipe_launch_n8(variant, conv, dtype, pa, r, sms, t, stream);
  if (n == 16) return pipe_launch_n16(variant, conv, dtype, pa, r, sms, t, stream);
  return pipe_launch_n32(variant, conv, dtype, pa, r, sms, t, stream);
}

// Apply one of the library's 1-D operators to every unit vector (host side).
template <int N, class P>
void build_int_matrices(double* T, double* U) {
  for (int j = 0; j < N; ++j) {
    int x[N], w[N];
    for (int i = 0; i < N; ++i) x[i] = w[i] = (i == j);
    Jam<N, P>::T(x);
    Jam<N, P>::W(w);  // 2 U
    for (int i = 0; i < N; ++i) {
      T[i * N + j] = x[i];
      U[i * N + j] = w[i] / 2;  // W = 2U is even: exact
    }
  }
}

void build_exact_matrices(double* T, double* U) {
  for (int j = 0; j < 8; ++j) {
    float x[8], y[8];
    for (int i = 0; i < 8; ++i) x[i] = y[i] = (i == j) ? 1.f : 0.f;
    T8_apply<ParamsExact>(x);   // 2 C
    T8t_apply<ParamsExact>(y);  // 2 C^T
    for (int i = 0; i < 8; ++i) {
      T[i * 8 + j] = x[i];
      U[i * 8 + j] = 2.0 * y[i];  // N T^{-1} = 8 (2C)^{-1} = 4 C^T
    }
  }
}

KernelSet select_kernels(int n, int variant, int conv, int dtype) {
  if (variant == CDCT_EXACT) return kernels_exact8(dtype);
  if (n == 8) return kernels_n8(variant, conv, dtype);
  if (n == 16) return kernels_n16(variant, conv, dtype);
  return kernels_n32(variant, conv, dtype);
}

cdct_status check_image(const cdct_image* in, const char* what) {
  if (in == nullptr) return fail(CDCT_EINVAL, std::string(what) + ": null image descriptor");
  if (in->data == nullptr) return fail(CDCT_EINVAL, std::string(what) + ": null data pointer");
  if (in->dtype != CDCT_U8 && in->dtype != CDCT_I16) return fail(CDCT_EINVAL, std::string(what) + ": bad dtype");
  if (in->width < 1 || in->height < 1) return fail(CDCT_EINVAL, std::string(what) + ": width and height must be >= 1");
  if (in->pitch < in->width) return fail(CDCT_EINVAL, std::string(what) + ": pitch < width");
  if (in->batch < 1) return fail(CDCT_EINVAL, std::string(what) + ": batch must be >= 1");
  if (in->batch > 1 && in->batch_stride < in->pitch * in->height)
    return fail(CDCT_EINVAL, std::string(what) + ": batch_stride < pitch * height");
  return CDCT_OK;
}

cdct_status check_recon(const float* recon, int64_t pitch, int64_t bstride, int width, int height, int batch) {
  if (recon == nullptr) return fail(CDCT_EINVAL, "null reconstruction pointer");
  if (pitch < width) return fail(CDCT_EINVAL, "recon_pitch < width");
  if (batch > 1 && bstride < pitch * height) return fail(CDCT_EINVAL, "recon_batch_stride < recon_pitch * height");
  return CDCT_OK;
}

// Geometry shared by the block kernels.
void fill_geometry(const cdct_plan_s* p, int width, int height, BlockArgs& a) {
  const int n = p->n;
  a.width = width;
  a.height = height;
  a.nbx = (width + n - 1) / n;
  a.nby = (height + n - 1) / n;
  a.blocks_per_img = static_cast<long long>(a.nbx) * a.nby;
  const int bpc = blocks_per_cta(n);
  a.ctas_per_img = static_cast<int>((a.blocks_per_img + bpc - 1) / bpc);
}

void fill_mask(const cdct_plan_s* p, int r, BlockArgs& a) {
  const int n = p->n, w = rows_per_thread(n), np = threads_per_block(n);
  for (int s = 0; s < 16; ++s) a.slab_mask[s] = 0ull;
  for (int s = 0; s < np; ++s)
    for (int k = 0; k < w; ++k)
      for (int i = 0; i < n; ++i)
        if (zigzag_pos(n, i, s * w + k) < r) a.slab_mask[s] |= 1ull << (k * n + i);
}

void fill_input(const cdct_image* in, BlockArgs& a) {
  const int es = in->dtype == CDCT_I16 ? 2 : 1;
  a.in = in->data;
  a.in_pitch = in->pitch;
  a.in_bstride = in->batch > 1 ? in->batch_stride : 0;
  a.in_vec = aligned16(in->data) && (in->pitch * es) % 16 == 0 &&
             (in->batch == 1 || (in->batch_stride * es) % 16 == 0);
}

void fill_output(float* recon, int64_t pitch, int64_t bstride, int batch, BlockArgs& a) {
  a.out = recon;
  a.out_pitch = pitch;
  a.out_bstride = batch > 1 ? bstride : 0;
  a.out_vec = aligned16(recon) && (pitch * 4) % 16 == 0 && (batch == 1 || (bstride * 4) % 16 == 0);
  a.out_v8 = (reinterpret_cast<uintptr_t>(recon) & 31u) == 0 && (pitch * 4) % 32 == 0 &&
             (batch == 1 || (bstride * 4) % 32 == 0);
}

// pipelined-kernel work units: segments of up to blocks_per_cta(n) blocks
long long units_per_row(const cdct_plan_s* p, const BlockArgs& a) {
  const int s = blocks_per_cta(p->n);
  return (a.nbx + s - 1) / s;
}

size_t partial_count(const cdct_plan_s* p, int width, int height, int batch) {
  BlockArgs a;
  fill_geometry(p, width, height, a);
  long long per = std::max<long long>(a.ctas_per_img, psnr_parts_per_img(height));
  per = std::max<long long>(per, units_per_row(p, a) * a.nby * (kThreads / 32));
  return static_cast<size_t>(per) * batch;
}

// scale from the integer kernel result to pixels: fused 4Z; inverse-only 2Z (paper) / 4Z
float recon_scale(const cdct_plan_s* p, bool fused) {
  if (p->variant == CDCT_EXACT) return fused ? 1.f / 16.f : 1.f / 4.f;
  const int mult = (fused || p->conv == 1) ? 4 : 2;
  return 1.f / static_cast<float>(mult * p->n * p->n);
}

}  // namespace

extern "C" {

const char* cdct_last_error(void) { return g_err.c_str(); }

const char* cdct_version(void) { return "cdct 0.1.0 (sm_103a)"; }

cdct_status cdct_plan_create(int n, int variant, uint32_t flags, cdct_plan* out) {
  if (out == nullptr) return fail(CDCT_EINVAL, "null output plan pointer");
  *out = nullptr;
  if (n != 8 && n != 16 && n != 32) return fail(CDCT_EINVAL, "n must be 8, 16 or 32");
  if (variant != CDCT_EXACT && variant != CDCT_TILDE && variant != CDCT_HAT)
    return fail(CDCT_EINVAL, "unknown variant");
  if (flags & ~CDCT_CONV_TRANSPOSE) return fail(CDCT_EINVAL, "unknown flag bits");
  if (variant == CDCT_EXACT && n != 8)
    return fail(CDCT_EUNSUPPORTED, "the exact DCT variant is provided for n = 8 only");
  cdct_plan_s* p = new (std::nothrow) cdct_plan_s();
  if (p == nullptr) return fail(CDCT_ENOMEM, "plan allocation failed");
  p->n = n;
  p->tuning.stages = 0;
  p->tuning.ctas_per_sm = 0;
  p->variant = variant;
  p->conv = (flags & CDCT_CONV_TRANSPOSE) ? 1 : 0;
  if (variant == CDCT_EXACT) build_exact_matrices(p->T, p->U);
  else if (variant == CDCT_TILDE) {
    if (n == 8) build_int_matrices<8, ParamsTilde>(p->T, p->U);
    else if (n == 16) build_int_matrices<16, ParamsTilde>(p->T, p->U);
    else build_int_matrices<32, ParamsTilde>(p->T, p->U);
  } else {
    if (n == 8) build_int_matrices<8, ParamsHat>(p->T, p->U);
    else if (n == 16) build_int_matrices<16, ParamsHat>(p->T, p->U);
    else build_int_matrices<32, ParamsHat>(p->T, p->U);
  }
  for (int i = 0; i < n; ++i) {
    double d = 0.0;
    for (int j = 0; j < n; ++j) d += p->T[i * n + j] * p->T[i * n + j];
    p->S[i] = 1.0 / std::sqrt(d);
    p->s_f[i] = static_cast<float>(p->S[i]);
  }
  p->ks[0] = select_kernels(n, variant, p->conv, 0);
  p->ks[1] = select_kernels(n, variant, p->conv, 1);
  *out = p;
  return CDCT_OK;
}

cdct_status cdct_plan_destroy(cdct_plan plan) {
  delete plan;
  return CDCT_OK;
}

cdct_status cdct_block_count(cdct_plan plan, const cdct_image* in, int64_t* n_blocks) {
  if (plan == nullptr || n_blocks == nullptr) return fail(CDCT_EINVAL, "null argument");
  cdct_status st = check_image(in, "block_count");
  if (st != CDCT_OK) return st;
  BlockArgs a;
  fill_geometry(plan, in->width, in->height, a);
  *n_blocks = a.blocks_per_img * in->batch;
  return CDCT_OK;
}

cdct_status cdct_workspace_size(cdct_plan plan, const cdct_image* in, size_t* bytes) {
  if (plan == nullptr || bytes == nullptr) return fail(CDCT_EINVAL, "null argument");
  cdct_status st = check_image(in, "workspace_size");
  if (st != CDCT_OK) return st;
  *bytes = partial_count(plan, in->width, in->height, in->batch) * sizeof(double);
  return CDCT_OK;
}

cdct_status cdct_forward(cdct_plan plan, const cdct_image* in, void* coeff, void* stream) {
  if (plan == nullptr) return fail(CDCT_EINVAL, "null plan");
  cdct_status st = check_image(in, "forward");
  if (st != CDCT_OK) return st;
  if (coeff == nullptr || !aligned16(coeff)) return fail(CDCT_EINVAL, "coeff must be a 16-byte aligned device pointer");
  BlockArgs a;
  std::memset(&a, 0, sizeof(a));
  fill_geometry(plan, in->width, in->height, a);
  fill_input(in, a);
  a.coeff = coeff;
  const int rc = plan->ks[in->dtype].forward(a, in->batch, stream);
  return rc ? cuda_fail(rc, "forward launch") : CDCT_OK;
}

cdct_status cdct_zonal(cdct_plan plan, int r, void* coeff, int64_t n_blocks, float* scaled, void* kept,
                       void* stream) {
  if (plan == nullptr || coeff == nullptr) return fail(CDCT_EINVAL, "null argument");
  if (r < 1 || r > plan->n * plan->n) return fail(CDCT_EINVAL, "r must be in [1, N*N]");
  if (n_blocks < 0) return fail(CDCT_EINVAL, "n_blocks < 0");
  const int rc = launch_zonal(plan->n, plan->variant == CDCT_EXACT, plan->conv, plan->s_f, r, coeff, n_blocks,
                              scaled, kept, stream);
  return rc ? cuda_fail(rc, "zonal launch") : CDCT_OK;
}

cdct_status cdct_inverse(cdct_plan plan, const void* coeff, int32_t width, int32_t height, int32_t batch,
                         float* recon, int64_t recon_pitch, int64_t recon_batch_stride, void* stream) {
  if (plan == nullptr) return fail(CDCT_EINVAL, "null plan");
  if (coeff == nullptr || !aligned16(coeff)) return fail(CDCT_EINVAL, "coeff must be a 16-byte aligned device pointer");
  if (width < 1 || height < 1 || batch < 1) return fail(CDCT_EINVAL, "width, height and batch must be >= 1");
  cdct_status st = check_recon(recon, recon_pitch, recon_batch_stride, width, height, batch);
  if (st != CDCT_OK) return st;
  BlockArgs a;
  std::memset(&a, 0, sizeof(a));
  fill_geometry(plan, width, height, a);
  a.coeff = const_cast<void*>(coeff);
  a.in = coeff;  // never dereferenced as pixels by the inverse kernels
  fill_output(recon, recon_pitch, recon_batch_stride, batch, a);
  a.scale = recon_scale(plan, false);
  const int rc = plan->ks[0].inverse(a, batch, stream);
  return rc ? cuda_fail(rc, "inverse launch") : CDCT_OK;
}

cdct_status cdct_psnr(const cdct_image* ref, const float* recon, int64_t recon_pitch, int64_t recon_batch_stride,
                      double* psnr_db, void* workspace, size_t workspace_bytes, void* stream) {
  cdct_status st = check_image(ref, "psnr");
  if (st != CDCT_OK) return st;
  st = check_recon(recon, recon_pitch, recon_batch_stride, ref->width, ref->height, ref->batch);
  if (st != CDCT_OK) return st;
  if (psnr_db == nullptr) return fail(CDCT_EINVAL, "null psnr output");
  const int parts = psnr_parts_per_img(ref->height);
  const size_t need = static_cast<size_t>(parts) * ref->batch * sizeof(double);
  if (workspace == nullptr || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 7u))
    return fail(CDCT_EINVAL, "workspace missing, misaligned or smaller than cdct_workspace_size()");
  double* partial = static_cast<double*>(workspace);
  int rc = launch_psnr_partials(ref->data, ref->dtype, ref->pitch, ref->batch > 1 ? ref->batch_stride : 0, recon,
                                recon_pitch, ref->batch > 1 ? recon_batch_stride : 0, ref->width, ref->height,
                                ref->batch, partial, parts, stream);
  if (rc) return cuda_fail(rc, "psnr launch");
  FinalArgs f;
  f.partial = partial;
  f.parts_per_img = parts;
  f.npix = static_cast<long long>(ref->width) * ref->height;
  f.psnr = psnr_db;
  f.sse = nullptr;
  rc = launch_finalize(f, ref->batch, stream);
  return rc ? cuda_fail(rc, "psnr finalize launch") : CDCT_OK;
}

cdct_status cdct_ssim_workspace_size(const cdct_image* ref, size_t* bytes) {
  cdct_status st = check_image(ref, "ssim");
  if (st != CDCT_OK) return st;
  if (bytes == nullptr) return fail(CDCT_EINVAL, "null bytes pointer");
  if (ref->width < 11 || ref->height < 11) return fail(CDCT_EINVAL, "ssim: images must be at least 11 x 11");
  *bytes = static_cast<size_t>(ssim_tiles(ref->width, ref->height)) * ref->batch * sizeof(double);
  return CDCT_OK;
}

cdct_status cdct_ssim(const cdct_image* ref, const float* recon, int64_t recon_pitch, int64_t recon_batch_stride,
                      double* ssim, void* workspace, size_t workspace_bytes, void* stream) {
  size_t need = 0;
  cdct_status st = cdct_ssim_workspace_size(ref, &need);
  if (st != CDCT_OK) return st;
  st = check_recon(recon, recon_pitch, recon_batch_stride, ref->width, ref->height, ref->batch);
  if (st != CDCT_OK) return st;
  if (ssim == nullptr) return fail(CDCT_EINVAL, "null ssim output");
  if (workspace == nullptr || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 7u))
    return fail(CDCT_EINVAL, "workspace missing, misaligned or smaller than cdct_ssim_workspace_size()");
  const int rc = ssim_launch(ref->data, ref->dtype, ref->pitch, ref->batch > 1 ? ref->batch_stride : 0, recon,
                             recon_pitch, ref->batch > 1 ? recon_batch_stride : 0, ref->width, ref->height,
                             ref->batch, static_cast<double*>(workspace), ssim, stream);
  return rc ? cuda_fail(rc, "ssim launch") : CDCT_OK;
}

cdct_status cdct_fwd_zonal_inv(cdct_plan plan, const cdct_image* in, int r, float* recon, int64_t recon_pitch,
                               int64_t recon_batch_stride, void* kept, double* psnr_db, void* workspace,
                               size_t workspace_bytes, void* stream) {
  if (plan == nullptr) return fail(CDCT_EINVAL, "null plan");
  cdct_status st = check_image(in, "fwd_zonal_inv");
  if (st != CDCT_OK) return st;
  if (r < 1 || r > plan->n * plan->n) return fail(CDCT_EINVAL, "r must be in [1, N*N]");
  st = check_recon(recon, recon_pitch, recon_batch_stride, in->width, in->height, in->batch);
  if (st != CDCT_OK) return st;
  if (kept != nullptr && (reinterpret_cast<uintptr_t>(kept) & 3u)) return fail(CDCT_EINVAL, "kept must be 4-byte aligned");
  BlockArgs a;
  std::memset(&a, 0, sizeof(a));
  fill_geometry(plan, in->width, in->height, a);
  fill_input(in, a);
  fill_output(recon, recon_pitch, recon_batch_stride, in->batch, a);
  fill_mask(plan, r, a);
  a.r = r;
  a.kept = kept;
  a.scale = recon_scale(plan, true);
  const int es = in->dtype == CDCT_I16 ? 2 : 1;
  const bool pipe = plan->variant != CDCT_EXACT && a.in_vec && (static_cast<long long>(in->width) * es) % 16 == 0 &&
                    units_per_row(plan, a) * a.nby * in->batch * (kThreads / 32) < (1ll << 31);
  PipeArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  long long parts_per_img = a.ctas_per_img;
  if (pipe) {
    pa.units_per_row = static_cast<int>(units_per_row(plan, a));
    pa.units_per_img = static_cast<long long>(pa.units_per_row) * a.nby;
    pa.total_units = pa.units_per_img * in->batch;
    pa.drop_copies = fault_mode(&pa.wait_limit) & 1;
    pa.div_img = make_fastdiv(static_cast<uint32_t>(pa.units_per_img));
    pa.div_row = make_fastdiv(static_cast<uint32_t>(pa.units_per_row));
    parts_per_img = pa.units_per_img * (kThreads / 32);   // one partial per warp and unit
    // the pipelined kernel masks 8 x 8 sub-blocks of the folded block
    const int nsub = (plan->n / 8) * (plan->n / 8);
    for (int q = 0; q < 16; ++q) a.slab_mask[q] = q < nsub ? sub_mask(plan->n, r, q) : 0ull;
  }
  if (psnr_db != nullptr) {
    const size_t need = static_cast<size_t>(parts_per_img) * in->batch * sizeof(double);
    if (workspace == nullptr || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 7u))
      return fail(CDCT_EINVAL, "workspace missing, misaligned or smaller than cdct_workspace_size()");
    a.partial = static_cast<double*>(workspace);
  }
  int rc;
  if (pipe) {
    DeviceInfo* di = nullptr;
    rc = device_info(&di);
    if (rc) return cuda_fail(rc, "device query");
    pa.b = a;
    pa.err = di->err;
    rc = pipe_launch(plan->n, plan->variant, plan->conv, in->dtype, pa, r, di->sms, plan->tuning, stream);
  } else {
    rc = plan->ks[in->dtype].fused(a, in->batch, stream);
  }
  if (rc) return cuda_fail(rc, "fused launch");
  if (psnr_db != nullptr) {
    FinalArgs f;
    f.partial = a.partial;
    f.parts_per_img = static_cast<int>(parts_per_img);
    f.npix = static_cast<long long>(in->width) * in->height;
    f.psnr = psnr_db;
    f.sse = nullptr;
    rc = launch_finalize(f, in->batch, stream);
    if (rc) return cuda_fail(rc, "psnr finalize launch");
  }
  return CDCT_OK;
}

cdct_status cdct_fwd_zonal_inv_noalloc(cdct_plan plan, const cdct_image* in, int r, float* recon,
                                       int64_t recon_pitch, int64_t recon_batch_stride, void* kept, double* psnr_db,
                                       void* stream) {
  if (plan == nullptr) return fail(CDCT_EINVAL, "null plan");
  cdct_status st = check_image(in, "fwd_zonal_inv_noalloc");
  if (st != CDCT_OK) return st;
  size_t need = 0;
  if (psnr_db != nullptr) {
    need = partial_count(plan, in->width, in->height, in->batch) * sizeof(double);
    if (need > kNoAllocScratchDoubles * sizeof(double))
      return fail(CDCT_EINVAL, "fwd_zonal_inv_noalloc: this call needs " + std::to_string(need) +
                                   " bytes of error partials, more than the fixed " +
                                   std::to_string(kNoAllocScratchDoubles * sizeof(double)) +
                                   "-byte scratch; use cdct_fwd_zonal_inv with a workspace");
  }
  // set-up, once per device with that device current: the scratch's device address
  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(static_cast<int>(e), "cudaGetDevice");
  if (dev < 0 || dev >= kMaxDevices) return fail(CDCT_EUNSUPPORTED, "device ordinal out of range");
  DeviceInfo& d = g_dev[dev];
  if (!d.scratch_ready.load(std::memory_order_acquire)) {
    std::lock_guard<std::mutex> lock(g_dev_mutex);
    if (!d.scratch_ready.load(std::memory_order_relaxed)) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(static_cast<int>(e), "cudaGetSymbolAddress(scratch)");
      d.noalloc_scratch = static_cast<double*>(ptr);
      d.scratch_ready.store(true, std::memory_order_release);
    }
  }
  // every partial a call reads is written by the same call, so the scratch
  // needs no clearing between calls
  return cdct_fwd_zonal_inv(plan, in, r, recon, recon_pitch, recon_batch_stride, kept, psnr_db, d.noalloc_scratch,
                            kNoAllocScratchDoubles * sizeof(double), stream);
}

cdct_status cdct_plan_set_tuning(cdct_plan plan, int stages, int ctas_per_sm) {
  if (plan == nullptr) return fail(CDCT_EINVAL, "null plan");
  if (stages < 0 || stages > 3) return fail(CDCT_EINVAL, "stages must be 0 (default), 1, 2 or 3");
  if (ctas_per_sm < 0 || ctas_per_sm > 32) return fail(CDCT_EINVAL, "ctas_per_sm must be in [0, 32]");
  plan->tuning.stages = stages;
  plan->tuning.ctas_per_sm = ctas_per_sm;
  return CDCT_OK;
}

cdct_status cdct_batch_create(cdct_plan plan, const cdct_batch_image* images, int n_images, int dtype,
                              cdct_batch* out) {
  if (out == nullptr) return fail(CDCT_EINVAL, "null output batch pointer");
  *out = nullptr;
  if (plan == nullptr || images == nullptr) return fail(CDCT_EINVAL, "null argument");
  if (plan->variant == CDCT_EXACT) return fail(CDCT_EUNSUPPORTED, "batches run the integer variants only");
  if (n_images < 1) return fail(CDCT_EINVAL, "n_images must be >= 1");
  if (dtype != CDCT_U8 && dtype != CDCT_I16) return fail(CDCT_EINVAL, "bad dtype");
  static_assert(sizeof(BatchImage) == sizeof(cdct_batch_image), "descriptor layout");
  static_assert(sizeof(UnitDesc) == 64, "unit descriptor layout");
  const int es = dtype == CDCT_I16 ? 2 : 1;
  const int n = plan->n, S = blocks_per_cta(n);
  std::vector<long long> prefix;
  try {
    prefix.resize(static_cast<size_t>(n_images) + 1);
  } catch (...) {
    return fail(CDCT_ENOMEM, "batch table allocation failed");
  }
  long long units = 0, pixels = 0;
  for (int i = 0; i < n_images; ++i) {
    const cdct_batch_image& im = images[i];
    const std::string where = "batch image " + std::to_string(i) + ": ";
    if (im.data == nullptr || im.recon == nullptr) return fail(CDCT_EINVAL, where + "null pointer");
    if (im.width < 1 || im.height < 1) return fail(CDCT_EINVAL, where + "width and height must be >= 1");
    if (im.pitch < im.width || im.recon_pitch < im.width) return fail(CDCT_EINVAL, where + "pitch < width");
    if (!aligned16(im.data) || !aligned16(im.recon) || (im.pitch * es) % 16 || (im.recon_pitch * 4) % 16 ||
        (static_cast<long long>(im.width) * es) % 16)
      return fail(CDCT_EINVAL, where + "pixels, rows and widths must be 16-byte aligned");
    prefix[i] = units;
    const long long nbx = (im.width + n - 1) / n, nby = (im.height + n - 1) / n;
    const int pack = pack_rows(static_cast<int>(nbx), S);
    units += pack > 1 ? (nby + pack - 1) / pack : nby * ((nbx + S - 1) / S);
    pixels += static_cast<long long>(im.width) * im.height;
  }
  prefix[n_images] = units;
  if (units * (kThreads / 32) >= (1ll << 31)) return fail(CDCT_EINVAL, "batch too large for one launch (2^31 work units)");
  // table: descriptors, unit prefix sums, then one UnitDesc per work unit
  const size_t desc_bytes = sizeof(BatchImage) * static_cast<size_t>(n_images);
  const size_t prefix_offset = (desc_bytes + 15) / 16 * 16;
  const size_t map_offset = (prefix_offset + sizeof(long long) * (static_cast<size_t>(n_images) + 1) + 15) / 16 * 16;
  const size_t table_bytes = map_offset + sizeof(UnitDesc) * static_cast<size_t>(units);
  cdct_batch_s* b = new (std::nothrow) cdct_batch_s();
  if (b == nullptr) return fail(CDCT_ENOMEM, "batch allocation failed");
  try {
    b->host_table.assign(table_bytes, '\0');
  } catch (...) {
    delete b;
    return fail(CDCT_ENOMEM, "batch table allocation failed");
  }
  std::memcpy(&b->host_table[prefix_offset], prefix.data(), sizeof(long long) * prefix.size());
  UnitDesc* map = reinterpret_cast<UnitDesc*>(&b->host_table[map_offset]);
  for (int i = 0; i < n_images; ++i) {
    const int nbx = (images[i].width + n - 1) / n, nby = (images[i].height + n - 1) / n;
    const int pack = pack_rows(nbx, S), upr = (nbx + S - 1) / S;
    for (long long k = 0; k < prefix[i + 1] - prefix[i]; ++k) {
      UnitDesc& m = map[prefix[i] + k];
      m.data = images[i].data;
      m.recon = images[i].recon;
      m.pitch = images[i].pitch;
      m.recon_pitch = images[i].recon_pitch;
      m.width = images[i].width;
      m.height = images[i].height;
      m.img = i;
      if (pack > 1) {
        m.by = static_cast<int32_t>(k * pack);
        m.seg = 0;
        m.rows = std::min(pack, nby - m.by);
      } else {
        m.by = static_cast<int32_t>(k / upr);
        m.seg = static_cast<int32_t>(k - static_cast<long long>(m.by) * upr);
        m.rows = 1;
      }
    }
  }
  std::memcpy(&b->host_table[0], images, desc_bytes);
  b->plan = plan;
  b->dtype = dtype;
  b->n_images = n_images;
  b->total_units = units;
  b->total_pixels = pixels;
  b->table_bytes = table_bytes;
  b->prefix_offset = prefix_offset;
  b->map_offset = map_offset;
  *out = b;
  return CDCT_OK;
}

cdct_status cdct_batch_destroy(cdct_batch batch) {
  delete batch;
  return CDCT_OK;
}

cdct_status cdct_batch_sizes(cdct_batch batch, size_t* table_bytes, size_t* workspace_bytes, int64_t* total_pixels) {
  if (batch == nullptr) return fail(CDCT_EINVAL, "null batch");
  if (table_bytes) *table_bytes = batch->table_bytes;
  if (workspace_bytes) *workspace_bytes = static_cast<size_t>(batch->total_units) * (kThreads / 32) * sizeof(double);
  if (total_pixels) *total_pixels = batch->total_pixels;
  return CDCT_OK;
}

cdct_status cdct_batch_unit(cdct_batch batch, int64_t unit, int32_t out[4]) {
  if (batch == nullptr || out == nullptr) return fail(CDCT_EINVAL, "null argument");
  if (unit < 0 || unit >= batch->total_units) return fail(CDCT_EINVAL, "unit out of range");
  const UnitDesc* map = reinterpret_cast<const UnitDesc*>(batch->host_table.data() + batch->map_offset);
  out[0] = map[unit].img;
  out[1] = map[unit].by;
  out[2] = map[unit].seg;
  out[3] = map[unit].rows;
  return CDCT_OK;
}

cdct_status cdct_batch_upload(cdct_batch batch, void* device_table, void* stream) {
  if (batch == nullptr || device_table == nullptr) return fail(CDCT_EINVAL, "null argument");
  if (!aligned16(device_table)) return fail(CDCT_EINVAL, "device_table must be 16-byte aligned");
  cudaError_t e = cudaMemcpyAsync(device_table, batch->host_table.data(), batch->table_bytes, cudaMemcpyHostToDevice,
                                  static_cast<cudaStream_t>(stream));
  if (e != cudaSuccess) return cuda_fail(static_cast<int>(e), "batch table upload");
  // the host copy is pageable: wait until it has been read
  e = cudaStreamSynchronize(static_cast<cudaStream_t>(stream));
  return e == cudaSuccess ? CDCT_OK : cuda_fail(static_cast<int>(e), "batch table upload");
}

cdct_status cdct_batch_fzi(cdct_batch batch, const void* device_table, int r, double* psnr_db, void* workspace,
                           size_t workspace_bytes, void* stream) {
  if (batch == nullptr || device_table == nullptr) return fail(CDCT_EINVAL, "null argument");
  const cdct_plan_s* plan = batch->plan;
  if (r < 1 || r > plan->n * plan->n) return fail(CDCT_EINVAL, "r must be in [1, N*N]");
  if (!aligned16(device_table)) return fail(CDCT_EINVAL, "device_table must be 16-byte aligned");
  const size_t need = static_cast<size_t>(batch->total_units) * (kThreads / 32) * sizeof(double);
  if (psnr_db != nullptr &&
      (workspace == nullptr || workspace_bytes < need || (reinterpret_cast<uintptr_t>(workspace) & 7u)))
    return fail(CDCT_EINVAL, "workspace missing, misaligned or smaller than cdct_batch_sizes()");
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return cuda_fail(rc, "device query");
  PipeArgs pa;
  std::memset(&pa, 0, sizeof(pa));
  BlockArgs& a = pa.b;
  a.out_vec = 1;
  a.r = r;
  a.scale = recon_scale(plan, true);
  a.partial = psnr_db != nullptr ? static_cast<double*>(workspace) : nullptr;
  const int nsub = (plan->n / 8) * (plan->n / 8);
  for (int q = 0; q < 16; ++q) a.slab_mask[q] = q < nsub ? sub_mask(plan->n, r, q) : 0ull;
  pa.total_units = batch->total_units;
  pa.drop_copies = fault_mode(&pa.wait_limit) & 1;
  pa.err = di->err;
  const BatchImage* images = static_cast<const BatchImage*>(device_table);
  const long long* unit_prefix =
      reinterpret_cast<const long long*>(static_cast<const char*>(device_table) + batch->prefix_offset);
  pa.unit_map = reinterpret_cast<const UnitDesc*>(static_cast<const char*>(device_table) + batch->map_offset);
  rc = pipe_launch(plan->n, plan->variant, plan->conv, batch->dtype, pa, r, di->sms, plan->tuning, stream);
  if (rc) return cuda_fail(rc, "batch launch");
  if (psnr_db != nullptr) {
    rc = launch_finalize_table(a.partial, unit_prefix, images, batch->n_images, kThreads / 32, psnr_db, stream);
    if (rc) return cuda_fail(rc, "batch psnr launch");
  }
  return CDCT_OK;
}

cdct_status cdct_set_fault_injection(int mode, int64_t wait_limit_cycles) {
  if (mode < 0 || mode > 3) return fail(CDCT_EINVAL, "fault injection mode must be 0..3");
  if (mode != 0 && (wait_limit_cycles < 1000 || wait_limit_cycles > kDefaultWaitLimit))
    return fail(CDCT_EINVAL, "fault injection wait limit must be in [1000, 2^31] cycles");
  g_fault_limit.store(mode ? wait_limit_cycles : kDefaultWaitLimit);
  g_fault_mode.store(mode);
  return CDCT_OK;
}

cdct_status cdct_check_device(void* stream) {
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return cuda_fail(rc, "device query");
  rc = static_cast<int>(cudaStreamSynchronize(static_cast<cudaStream_t>(stream)));
  if (rc) return cuda_fail(rc, "stream synchronize");
  int word = 0;
  rc = static_cast<int>(cudaMemcpy(&word, di->err, sizeof(int), cudaMemcpyDeviceToHost));
  if (rc) return cuda_fail(rc, "error word read");
  if (word == 0) return CDCT_OK;
  const int zero = 0;
  rc = static_cast<int>(cudaMemcpy(di->err, &zero, sizeof(int), cudaMemcpyHostToDevice));
  if (rc) return cuda_fail(rc, "error word reset");
  return fail(CDCT_ETIMEOUT, (word & 1) ? "a kernel gave up waiting for its staged input (bounded wait expired)"
                                        : "a kernel gave up waiting for its tensor-core products (bounded wait expired)");
}

cdct_status cdct_rd_create(int variant, cdct_rd* out) {
  if (out == nullptr) return fail(CDCT_EINVAL, "null output handle");
  *out = nullptr;
  if (variant != CDCT_TILDE && variant != CDCT_HAT)
    return fail(CDCT_EINVAL, "the rate-distortion search needs CDCT_TILDE or CDCT_HAT");
  cdct_rd_s* rd = new (std::nothrow) cdct_rd_s;
  if (rd == nullptr) return fail(CDCT_ENOMEM, "out of host memory");
  rd->variant = variant;
  if (rd_table_words() != static_cast<int>(sizeof(rd->tables) / sizeof(int))) {
    delete rd;
    return fail(CDCT_EUNSUPPORTED, "internal table size mismatch");
  }
  rd_tables(variant, rd->tables);
  *out = rd;
  return CDCT_OK;
}

cdct_status cdct_rd_destroy(cdct_rd rd) {
  delete rd;
  return CDCT_OK;
}

cdct_status cdct_rd_tables(cdct_rd rd, int32_t* out) {
  if (rd == nullptr || out == nullptr) return fail(CDCT_EINVAL, "null argument");
  std::memcpy(out, rd->tables, sizeof(rd->tables));
  return CDCT_OK;
}

cdct_status cdct_rd_region_count(const cdct_image* in, int64_t* n_regions) {
  if (n_regions == nullptr) return fail(CDCT_EINVAL, "null output");
  cdct_status st = check_image(in, "rd input");
  if (st != CDCT_OK) return st;
  *n_regions = static_cast<int64_t>(in->batch) * ((in->width + 31) / 32) * ((in->height + 31) / 32);
  return CDCT_OK;
}

namespace {
// argument checks shared by the RD entry points; lambda' per step as 128-bit words
cdct_status rd_common(cdct_rd rd, const cdct_image* in, const int32_t* q, int32_t n_q, int32_t kappa_num,
                      int32_t kappa_log2_den, int64_t* n_regions, unsigned long long* lo, unsigned long long* hi) {
  if (rd == nullptr) return fail(CDCT_EINVAL, "null rd handle");
  cdct_status st = cdct_rd_region_count(in, n_regions);
  if (st != CDCT_OK) return st;
  if (q == nullptr || n_q < 1 || n_q > 4) return fail(CDCT_EINVAL, "n_q must be 1..4 with a host array q");
  for (int k = 0; k < n_q; ++k)
    if (q[k] < 1 || q[k] > 4096) return fail(CDCT_EINVAL, "quantiser steps must be in 1..4096");
  if (kappa_num < 0 || kappa_num > 1024) return fail(CDCT_EINVAL, "kappa_num must be in 0..1024");
  if (kappa_log2_den < 0 || kappa_log2_den > 44) return fail(CDCT_EINVAL, "kappa_log2_den must be in 0..44");
  for (int k = 0; k < n_q; ++k) {
    const unsigned __int128 lam = static_cast<unsigned __int128>(static_cast<unsigned long long>(kappa_num) *
                                                                 static_cast<unsigned long long>(q[k]) * q[k])
                                  << (44 - kappa_log2_den);
    lo[k] = static_cast<unsigned long long>(lam);
    hi[k] = static_cast<unsigned long long>(lam >> 64);
  }
  return CDCT_OK;
}
}  // namespace

cdct_status cdct_rd_search(cdct_rd rd, const cdct_image* in, const int32_t* q, int32_t n_q, int32_t kappa_num,
                           int32_t kappa_log2_den, uint8_t* labels, uint64_t* partition_cost, void* stream) {
  int64_t n_regions = 0;
  unsigned long long lo[4], hi[4];
  cdct_status st = rd_common(rd, in, q, n_q, kappa_num, kappa_log2_den, &n_regions, lo, hi);
  if (st != CDCT_OK) return st;
  if (labels == nullptr) return fail(CDCT_EINVAL, "null labels pointer");
  if (n_regions == 0) return CDCT_OK;
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return cuda_fail(rc, "device query");
  rc = launch_rd(rd->variant, in->dtype, in->data, in->pitch, in->batch_stride, in->width, in->height, in->batch,
                 rd->tables, q, n_q, lo, hi, labels, reinterpret_cast<unsigned long long*>(partition_cost), di->sms,
                 stream);
  return rc ? cuda_fail(rc, "rd launch") : CDCT_OK;
}

cdct_status cdct_rd_search_subset(cdct_rd rd, const cdct_image* in, const int32_t* q, int32_t n_q,
                                  int32_t kappa_num, int32_t kappa_log2_den, const int64_t* region_index,
                                  const int64_t* count, int64_t max_count, uint8_t* labels,
                                  uint64_t* partition_cost, void* stream) {
  int64_t n_regions = 0;
  unsigned long long lo[4], hi[4];
  cdct_status st = rd_common(rd, in, q, n_q, kappa_num, kappa_log2_den, &n_regions, lo, hi);
  if (st != CDCT_OK) return st;
  if (labels == nullptr || region_index == nullptr || count == nullptr)
    return fail(CDCT_EINVAL, "null labels, region_index or count pointer");
  if (max_count < 0 || max_count > n_regions) return fail(CDCT_EINVAL, "max_count must be in 0..n_regions");
  if (max_count == 0) return CDCT_OK;
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return cuda_fail(rc, "device query");
  RdModeArgs m{};
  m.mode = 1;
  m.subset = reinterpret_cast<const long long*>(region_index);
  m.subset_count = reinterpret_cast<const long long*>(count);
  m.max_count = max_count;
  rc = launch_rd(rd->variant, in->dtype, in->data, in->pitch, in->batch_stride, in->width, in->height, in->batch,
                 rd->tables, q, n_q, lo, hi, labels, reinterpret_cast<unsigned long long*>(partition_cost), di->sms,
                 stream, &m);
  return rc ? cuda_fail(rc, "rd subset launch") : CDCT_OK;
}

cdct_status cdct_rd_evaluate(cdct_rd rd, const cdct_image* in, const int32_t* q, int32_t n_q, int32_t kappa_num,
                             int32_t kappa_log2_den, const uint8_t* labels, uint64_t* cost, uint64_t* dist,
                             int32_t* bits, void* stream) {
  int64_t n_regions = 0;
  unsigned long long lo[4], hi[4];
  cdct_status st = rd_common(rd, in, q, n_q, kappa_num, kappa_log2_den, &n_regions, lo, hi);
  if (st != CDCT_OK) return st;
  if (labels == nullptr || cost == nullptr) return fail(CDCT_EINVAL, "null labels or cost pointer");
  if (n_regions == 0) return CDCT_OK;
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return cuda_fail(rc, "device query");
  RdModeArgs m{};
  m.mode = 2;
  m.in_labels = labels;
  m.ev_cost = reinterpret_cast<unsigned long long*>(cost);
  m.ev_dist = reinterpret_cast<unsigned long long*>(dist);
  m.ev_bits = bits;
  rc = launch_rd(rd->variant, in->dtype, in->data, in->pitch, in->batch_stride, in->width, in->height, in->batch,
                 rd->tables, q, n_q, lo, hi, nullptr, nullptr, di->sms, stream, &m);
  return rc ? cuda_fail(rc, "rd evaluate launch") : CDCT_OK;
}

cdct_status cdct_cnn_select(const float* margin, int64_t n_regions, int32_t n_slots, float threshold,
                            int64_t* region_index, int64_t* count, void* stream) {
  if (margin == nullptr || region_index == nullptr || count == nullptr) return fail(CDCT_EINVAL, "null pointer argument");
  if (n_regions < 0) return fail(CDCT_EINVAL, "n_regions must be >= 0");
  if (n_slots < 1 || n_slots > CDCT_CNN_SLOTS) return fail(CDCT_EINVAL, "n_slots must be 1..4");
  if (std::isnan(threshold)) return fail(CDCT_EINVAL, "threshold is NaN");
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return cuda_fail(rc, "device query");
  rc = cnn_select_launch(margin, n_regions, n_slots, threshold, reinterpret_cast<long long*>(region_index),
                         reinterpret_cast<long long*>(count), di->sms, stream);
  return rc ? cuda_fail(rc, "cnn select launch") : CDCT_OK;
}

// ---- learned quadtree selector ----------------------------------------------

size_t cdct_cnn_packed_bytes(void) { return cnn::kPackedBytes; }

cdct_status cdct_cnn_pack(const float* params, void* packed, void* stream) {
  if (params == nullptr || packed == nullptr) return fail(CDCT_EINVAL, "null params or packed pointer");
  if (!aligned16(params) || !aligned16(packed)) return fail(CDCT_EINVAL, "params and packed must be 16-byte aligned");
  const int rc = cnn_pack_launch(params, packed, stream);
  return rc ? cuda_fail(rc, "cnn pack launch") : CDCT_OK;
}

namespace {
cdct_status check_slots(const int32_t* slots, int32_t n_slots) {
  if (slots == nullptr || n_slots < 1 || n_slots > CDCT_CNN_SLOTS)
    return fail(CDCT_EINVAL, "n_slots must be 1..4 with a host array of slots");
  for (int k = 0; k < n_slots; ++k)
    if (slots[k] < 0 || slots[k] >= CDCT_CNN_SLOTS) return fail(CDCT_EINVAL, "quantiser slots must be in 0..3");
  return CDCT_OK;
}
}  // namespace

cdct_status cdct_cnn_infer(const void* packed, const cdct_image* in, const int32_t* slots, int32_t n_slots,
                           uint8_t* labels, float* logits, float* margin, void* stream) {
  if (packed == nullptr || !aligned16(packed)) return fail(CDCT_EINVAL, "packed weights: null or not 16-byte aligned");
  int64_t n_regions = 0;
  cdct_status st = cdct_rd_region_count(in, &n_regions);
  if (st != CDCT_OK) return st;
  st = check_slots(slots, n_slots);
  if (st != CDCT_OK) return st;
  if (labels == nullptr) return fail(CDCT_EINVAL, "null labels pointer");
  if (n_regions >= (int64_t{1} << 31)) return fail(CDCT_EINVAL, "more than 2^31 - 1 regions in one call");
  if (n_regions == 0) return CDCT_OK;
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return cuda_fail(rc, "device query");
  int sl[CDCT_CNN_SLOTS];
  for (int k = 0; k < n_slots; ++k) sl[k] = slots[k];
  rc = cnn_infer_launch(packed, in->data, in->dtype, in->pitch, in->batch_stride, in->width, in->height, in->batch,
                        sl, n_slots, labels, logits, margin, di->sms, di->err, stream);
  return rc ? cuda_fail(rc, "cnn inference launch") : CDCT_OK;
}

cdct_status cdct_cnn_workspace_size(int32_t batch, size_t* bytes) {
  if (bytes == nullptr) return fail(CDCT_EINVAL, "null bytes pointer");
  if (batch < 64 || batch % 64 != 0) return fail(CDCT_EINVAL, "batch must be a positive multiple of 64");
  *bytes = cnn_train_workspace(batch);
  return CDCT_OK;
}

cdct_status cdct_cnn_grad(const float* params, const int16_t* regions, int32_t batch, const int32_t* slots,
                          int32_t n_slots, const uint8_t* labels, const uint64_t* partition_cost, float mu,
                          float* grad, float* loss, void* workspace, size_t workspace_bytes, void* stream) {
  if (params == nullptr || regions == nullptr || labels == nullptr || grad == nullptr || loss == nullptr ||
      workspace == nullptr)
    return fail(CDCT_EINVAL, "null pointer argument");
  if (batch < 64 || batch % 64 != 0) return fail(CDCT_EINVAL, "batch must be a positive multiple of 64");
  cdct_status st = check_slots(slots, n_slots);
  if (st != CDCT_OK) return st;
  if (!(mu >= 0.f) || !std::isfinite(mu)) return fail(CDCT_EINVAL, "mu must be finite and >= 0");
  if ((reinterpret_cast<uintptr_t>(workspace) & 255u) != 0) return fail(CDCT_EINVAL, "workspace must be 256-byte aligned");
  if (!aligned16(params) || !aligned16(grad)) return fail(CDCT_EINVAL, "params and grad must be 16-byte aligned");
  if (workspace_bytes < cnn_train_workspace(batch)) return fail(CDCT_EINVAL, "workspace too small");
  int sl[CDCT_CNN_SLOTS];
  for (int k = 0; k < n_slots; ++k) sl[k] = slots[k];
  DeviceInfo* di = nullptr;
  int rc = device_info(&di);
  if (rc) return cuda_fail(rc, "device query");
  rc = cnn_grad_launch(params, regions, batch, sl, n_slots, labels,
                       reinterpret_cast<const unsigned long long*>(partition_cost), mu, grad, loss, workspace, di->err,
                       stream);
  return rc ? cuda_fail(rc, "cnn gradient launch") : CDCT_OK;
}

cdct_status cdct_cnn_adam(float* params, const float* grad, float* m, float* v, int32_t step, float lr, float beta1,
                          float beta2, float eps, void* stream) {
  if (params == nullptr || grad == nullptr || m == nullptr || v == nullptr) return fail(CDCT_EINVAL, "null pointer argument");
  if (step < 1) return fail(CDCT_EINVAL, "step must be >= 1");
  if (!(lr > 0.f) || !std::isfinite(lr) || !(beta1 >= 0.f && beta1 < 1.f) || !(beta2 >= 0.f && beta2 < 1.f) ||
      !(eps > 0.f) || !std::isfinite(eps))
    return fail(CDCT_EINVAL, "need lr > 0, 0 <= beta1, beta2 < 1 and eps > 0");
  const int rc = cnn_adam_launch(params, grad, m, v, step, lr, beta1, beta2, eps, stream);
  return rc ? cuda_fail(rc, "adam launch") : CDCT_OK;
}

cdct_status cdct_matrix(cdct_plan plan, int which, double* out) {
  if (plan == nullptr || out == nullptr) return fail(CDCT_EINVAL, "null argument");
  const int n = plan->n;
  switch (which) {
    case CDCT_MATRIX_T: std::memcpy(out, plan->T, sizeof(double) * n * n); return CDCT_OK;
    case CDCT_MATRIX_U: std::memcpy(out, plan->U, sizeof(double) * n * n); return CDCT_OK;
    case CDCT_MATRIX_S: std::memcpy(out, plan->S, sizeof(double) * n); return CDCT_OK;
    case CDCT_MATRIX_ZIGZAG:
      for (int i = 0; i < n; ++i)
        for (int j = 0; j < n; ++j) out[i * n + j] = zigzag_pos(n, i, j);
      return CDCT_OK;
    default: return fail(CDCT_EINVAL, "unknown matrix selector");
  }
}

}  // extern "C"
