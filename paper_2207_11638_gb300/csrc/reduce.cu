// Elementwise zonal kernel, standalone error partials and the per-image
// SSE -> PSNR finalisation.  All reductions run in a fixed order, so the
// results are bit-reproducible from run to run.
#include <cuda_runtime.h>
#include <math.h>

#include "common.cuh"

namespace cdct {
namespace {

constexpr int kFinalThreads = 256;
constexpr int kPsnrRows = 4;           // image rows per CTA of the standalone error kernel

// psnr[img] = 10 log10(255^2 npix / SSE), +inf when SSE = 0 (Sec. 5.1 PSNR);
// NaN partials (a kernel that gave up a bounded wait) give NaN.
__global__ void __launch_bounds__(kFinalThreads) finalize_kernel(const FinalArgs a) {
  __shared__ double red[kFinalThreads];
  const int img = blockIdx.x;
  const double* part = a.partial + static_cast<long long>(img) * a.parts_per_img;
  double s = 0.0;
  for (int i = threadIdx.x; i < a.parts_per_img; i += kFinalThreads) s += part[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kFinalThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sse = red[0];
    if (a.sse != nullptr) a.sse[img] = sse;
    a.psnr[img] = (sse == 0.0) ? static_cast<double>(INFINITY)
                               : 10.0 * log10(255.0 * 255.0 * static_cast<double>(a.npix) / sse);
  }
}

// per-image PSNR of a descriptor-table batch: image i owns partials
// [unit_prefix[i] * W, unit_prefix[i + 1] * W), summed in a fixed order
__global__ void __launch_bounds__(kFinalThreads) finalize_table_kernel(const double* partial,
                                                                       const long long* unit_prefix,
                                                                       const BatchImage* images, int warps,
                                                                       double* psnr) {
  __shared__ double red[kFinalThreads];
  const int img = blockIdx.x;
  const long long b = unit_prefix[img] * warps, e = unit_prefix[img + 1] * warps;
  double s = 0.0;
  for (long long i = b + threadIdx.x; i < e; i += kFinalThreads) s += partial[i];
  red[threadIdx.x] = s;
  __syncthreads();
  for (int w = kFinalThreads / 2; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) {
    const double sse = red[0];
    const double npix = static_cast<double>(images[img].width) * images[img].height;
    psnr[img] = (sse == 0.0) ? static_cast<double>(INFINITY) : 10.0 * log10(255.0 * 255.0 * npix / sse);
  }
}

struct ZonalArgs {
  int n, exact, conv, r;
  void* coeff;
  long long total;        // nblocks * n * n
  float* scaled;
  void* kept;
  float s[32];            // diag(S_N)
  float inv_s[32];
};

// Ym = mask o Y in place; optional scaled B and kept coefficients (Sec. 5.1).
__global__ void zonal_kernel(const ZonalArgs a) {
  const long long e = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x;
  if (e >= a.total) return;
  const int nn = a.n * a.n;
  const long long blk = e / nn;
  const int w = static_cast<int>(e - blk * nn);
  const int i = w / a.n, j = w - (w / a.n) * a.n;
  const int pos = zigzag_pos(a.n, i, j);
  const bool keep = pos < a.r;
  float val;
  if (a.exact) {
    float* c = static_cast<float*>(a.coeff) + e;
    if (!keep) *c = 0.f;
    val = *c;
    if (keep && a.kept != nullptr) static_cast<float*>(a.kept)[blk * a.r + pos] = val;
  } else {
    int* c = static_cast<int*>(a.coeff) + e;
    if (!keep) *c = 0;
    if (keep && a.kept != nullptr) static_cast<int*>(a.kept)[blk * a.r + pos] = *c;
    val = static_cast<float>(*c);
  }
  if (a.scaled != nullptr) {
    // paper: B = diag(s) Y diag(s)^-1 / N ; transpose: B = diag(s) Y diag(s); exact: B itself
    float b;
    if (a.exact) b = val;
    else if (a.conv == 0) b = val * a.s[i] * a.inv_s[j] / static_cast<float>(a.n);
    else b = val * a.s[i] * a.s[j];
    a.scaled[e] = b;
  }
}

template <typename InT>
__global__ void __launch_bounds__(256) psnr_partial_kernel(const InT* ref, long long ref_pitch, long long ref_bstride,
                                                           const float* rec, long long rec_pitch, long long rec_bstride,
                                                           int width, int height, int parts_per_img, double* partial) {
  __shared__ double red[256];
  const int img = blockIdx.x / parts_per_img;
  const int part = blockIdx.x - img * parts_per_img;
  double total = 0.0;
  for (int rr = 0; rr < kPsnrRows; ++rr) {
    const int y = part * kPsnrRows + rr;
    if (y >= height) break;
    const InT* rrow = ref + img * ref_bstride + y * ref_pitch;
    const float* crow = rec + img * rec_bstride + y * rec_pitch;
    float acc = 0.f;
    for (int x = threadIdx.x; x < width; x += 256) {
      const float e = crow[x] - static_cast<float>(rrow[x]);
      acc = fmaf(e, e, acc);
    }
    total += static_cast<double>(acc);
  }
  red[threadIdx.x] = total;
  __syncthreads();
  for (int w = 128; w > 0; w >>= 1) {
    if (threadIdx.x < w) red[threadIdx.x] += red[threadIdx.x + w];
    __syncthreads();
  }
  if (threadIdx.x == 0) partial[blockIdx.x] = red[0];
}

}  // namespace

int launch_finalize(const FinalArgs& a, int batch, void* stream) {
  finalize_kernel<<<batch, kFinalThreads, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}

int launch_finalize_table(const double* partial, const long long* unit_prefix, const BatchImage* images,
                          int n_images, int warps_per_unit, double* psnr, void* stream) {
  finalize_table_kernel<<<n_images, kFinalThreads, 0, static_cast<cudaStream_t>(stream)>>>(
      partial, unit_prefix, images, warps_per_unit, psnr);
  return static_cast<int>(cudaGetLastError());
}

int launch_zonal(int n, int exact, int conv, const float* s, int r, void* coeff, long long nblocks,
                 float* scaled, void* kept, void* stream) {
  ZonalArgs a;
  a.n = n; a.exact = exact; a.conv = conv; a.r = r; a.coeff = coeff;
  a.total = nblocks * n * n; a.scaled = scaled; a.kept = kept;
  for (int i = 0; i < 32; ++i) { a.s[i] = i < n ? s[i] : 0.f; a.inv_s[i] = i < n ? 1.f / s[i] : 0.f; }
  if (a.total == 0) return 0;
  const long long grid = (a.total + 255) / 256;
  zonal_kernel<<<static_cast<unsigned>(grid), 256, 0, static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}

int psnr_parts_per_img(int height) { return (height + kPsnrRows - 1) / kPsnrRows; }

int launch_psnr_partials(const void* ref, int dtype, long long ref_pitch, long long ref_bstride,
                         const float* recon, long long rec_pitch, long long rec_bstride,
                         int width, int height, int batch, double* partial, int parts_per_img,
                         void* stream) {
  const dim3 grid(static_cast<unsigned>(batch) * parts_per_img);
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  if (dtype == 0)
    psnr_partial_kernel<uint8_t><<<grid, 256, 0, st>>>(static_cast<const uint8_t*>(ref), ref_pitch, ref_bstride,
                                                       recon, rec_pitch, rec_bstride, width, height, parts_per_img, partial);
  else
    psnr_partial_kernel<int16_t><<<grid, 256, 0, st>>>(static_cast<const int16_t*>(ref), ref_pitch, ref_bstride,
                                                       recon, rec_pitch, rec_bstride, width, height, parts_per_img, partial);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace cdct
