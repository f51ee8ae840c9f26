// Mean SSIM of reconstructions against their references, per image.
//
// The JPEG-like experiment of Sec. 5.1 compares reconstructions by PSNR and
// by the structural similarity index of Wang et al. (2004), which the paper
// cites without restating.  The standard form is used: an 11 x 11 circularly
// symmetric Gaussian window w (sigma 1.5, unit sum), K1 = 0.01, K2 = 0.03,
// L = 255, local statistics at every window position that lies inside the
// image, and the mean of the resulting map:
//   mu_x = sum w x,  s_xx = sum w x^2 - mu_x^2,  s_xy = sum w x y - mu_x mu_y, ...
//   SSIM = (2 mu_x mu_y + C1)(2 s_xy + C2) / ((mu_x^2 + mu_y^2 + C1)(s_xx + s_yy + C2)).
// The window is separable (w = g g^T), so each CTA filters a 32 x 32 tile of
// window positions in two passes through shared memory: rows (42 x 32 x 5
// sums), then columns.  The arithmetic is float64: the variance terms are
// differences of sums of squares of 8-bit values, where float32 would lose
// the low digits the index depends on in flat regions.  Each CTA writes one
// partial sum; a second kernel adds them per image in a fixed order.
#include <cuda_runtime.h>

#include <cmath>
#include <cstdint>

namespace cdct {
namespace {

constexpr int kWin = 11, kTile = 32, kHalo = kTile + kWin - 1;   // 42
constexpr int kSsimThreads = 256;

struct SsimArgs {
  const void* ref;
  int dtype;               // 0 u8, 1 i16
  long long ref_pitch, ref_bstride;
  const float* rec;
  long long rec_pitch, rec_bstride;
  int width, height;       // image size; window positions (height - 10) x (width - 10)
  int tiles_x, tiles_per_img;
  double g[kWin];          // 1-D Gaussian, sum 1
  double* partial;         // [batch][tiles_per_img]
};

template <typename InT>
__global__ void __launch_bounds__(kSsimThreads) ssim_tile_kernel(const SsimArgs a) {
  extern __shared__ __align__(16) double smem_ssim[];
  double (*sx)[kHalo] = reinterpret_cast<double (*)[kHalo]>(smem_ssim);
  double (*sy)[kHalo] = reinterpret_cast<double (*)[kHalo]>(smem_ssim + kHalo * kHalo);
  double (*hs)[kHalo][kTile] = reinterpret_cast<double (*)[kHalo][kTile]>(smem_ssim + 2 * kHalo * kHalo);  // mu_x, mu_y, xx, yy, xy
  __shared__ double red[kSsimThreads / 32];
  const int tid = threadIdx.x;
  const int img = blockIdx.x / a.tiles_per_img, t = blockIdx.x - img * a.tiles_per_img;
  const int ty = t / a.tiles_x, tx = t - ty * a.tiles_x;
  const int oy = ty * kTile, ox = tx * kTile;          // first window position of the tile
  const int mh = a.height - (kWin - 1), mw = a.width - (kWin - 1);
  const InT* ref = static_cast<const InT*>(a.ref) + img * a.ref_bstride;
  const float* rec = a.rec + img * a.rec_bstride;
  for (int i = tid; i < kHalo * kHalo; i += kSsimThreads) {
    const int r = i / kHalo, c = i - r * kHalo;
    const int gy = min(oy + r, a.height - 1), gx = min(ox + c, a.width - 1);   // clamped reads feed only unused positions
    sx[r][c] = static_cast<double>(ref[gy * a.ref_pitch + gx]);
    sy[r][c] = static_cast<double>(rec[gy * a.rec_pitch + gx]);
  }
  __syncthreads();
  for (int i = tid; i < kHalo * kTile; i += kSsimThreads) {
    const int r = i / kTile, c = i - r * kTile;
    double m1 = 0, m2 = 0, s11 = 0, s22 = 0, s12 = 0;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const double x = sx[r][c + k], y = sy[r][c + k], w = a.g[k];
      m1 += w * x;
      m2 += w * y;
      s11 += w * x * x;
      s22 += w * y * y;
      s12 += w * x * y;
    }
    hs[0][r][c] = m1;
    hs[1][r][c] = m2;
    hs[2][r][c] = s11;
    hs[3][r][c] = s22;
    hs[4][r][c] = s12;
  }
  __syncthreads();
  const double c1 = (0.01 * 255.0) * (0.01 * 255.0), c2 = (0.03 * 255.0) * (0.03 * 255.0);
  double acc = 0.0;
  for (int i = tid; i < kTile * kTile; i += kSsimThreads) {
    const int r = i / kTile, c = i - r * kTile;
    if (oy + r >= mh || ox + c >= mw) continue;
    double m1 = 0, m2 = 0, s11 = 0, s22 = 0, s12 = 0;
#pragma unroll
    for (int k = 0; k < kWin; ++k) {
      const double w = a.g[k];
      m1 += w * hs[0][r + k][c];
      m2 += w * hs[1][r + k][c];
      s11 += w * hs[2][r + k][c];
      s22 += w * hs[3][r + k][c];
      s12 += w * hs[4][r + k][c];
    }
    const double vx = s11 - m1 * m1, vy = s22 - m2 * m2, cxy = s12 - m1 * m2;
    acc += ((2 * m1 * m2 + c1) * (2 * cxy + c2)) / ((m1 * m1 + m2 * m2 + c1) * (vx + vy + c2));
  }
  for (int o = 16; o > 0; o >>= 1) acc += __shfl_down_sync(0xffffffffu, acc, o);
  if ((tid & 31) == 0) red[tid >> 5] = acc;
  __syncthreads();
  if (tid == 0) {
    double s = 0.0;
    for (int w = 0; w < kSsimThreads / 32; ++w) s += red[w];
    a.partial[blockIdx.x] = s;
  }
}

__global__ void ssim_finalize_kernel(const double* partial, int tiles_per_img, int batch, long long positions,
                                     double* ssim) {
  const int img = blockIdx.x * blockDim.x + threadIdx.x;
  if (img >= batch) return;
  double s = 0.0;
  for (int t = 0; t < tiles_per_img; ++t) s += partial[static_cast<long long>(img) * tiles_per_img + t];
  ssim[img] = s / static_cast<double>(positions);
}

}  // namespace

long long ssim_tiles(int width, int height) {
  const int mh = height - (kWin - 1), mw = width - (kWin - 1);
  return static_cast<long long>((mw + kTile - 1) / kTile) * ((mh + kTile - 1) / kTile);
}

int ssim_launch(const void* ref, int dtype, long long ref_pitch, long long ref_bstride, const float* rec,
                long long rec_pitch, long long rec_bstride, int width, int height, int batch, double* partial,
                double* ssim, void* stream) {
  SsimArgs a;
  a.ref = ref;
  a.dtype = dtype;
  a.ref_pitch = ref_pitch;
  a.ref_bstride = ref_bstride;
  a.rec = rec;
  a.rec_pitch = rec_pitch;
  a.rec_bstride = rec_bstride;
  a.width = width;
  a.height = height;
  a.tiles_x = (width - (kWin - 1) + kTile - 1) / kTile;
  a.tiles_per_img = static_cast<int>(ssim_tiles(width, height));
  double sum = 0.0;
  for (int k = 0; k < kWin; ++k) {
    const double d = k - (kWin - 1) / 2.0;
    a.g[k] = std::exp(-d * d / (2.0 * 1.5 * 1.5));
    sum += a.g[k];
  }
  for (int k = 0; k < kWin; ++k) a.g[k] /= sum;
  a.partial = partial;
  cudaStream_t s = static_cast<cudaStream_t>(stream);
  const long long ctas = static_cast<long long>(batch) * a.tiles_per_img;
  const int smem = static_cast<int>((2 * kHalo * kHalo + 5 * kHalo * kTile) * sizeof(double));
  cudaError_t e;
  if (dtype == 0) {
    e = cudaFuncSetAttribute(ssim_tile_kernel<uint8_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return static_cast<int>(e);
    ssim_tile_kernel<uint8_t><<<static_cast<unsigned>(ctas), kSsimThreads, smem, s>>>(a);
  } else {
    e = cudaFuncSetAttribute(ssim_tile_kernel<int16_t>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return static_cast<int>(e);
    ssim_tile_kernel<int16_t><<<static_cast<unsigned>(ctas), kSsimThreads, smem, s>>>(a);
  }
  e = cudaGetLastError();
  if (e != cudaSuccess) return static_cast<int>(e);
  const long long positions = static_cast<long long>(height - (kWin - 1)) * (width - (kWin - 1));
  ssim_finalize_kernel<<<(batch + 127) / 128, 128, 0, s>>>(partial, a.tiles_per_img, batch, positions, ssim);
  return static_cast<int>(cudaGetLastError());
}

}  // namespace cdct
