// Shared declarations of the CUDA library (not part of the public C ABI).
#pragma once
#include <cstdint>

namespace cdct {

constexpr int kThreads = 128;        // threads per CTA of the block kernels

// Launch arguments of the block kernels (fused, forward, inverse).
struct BlockArgs {
  // input image batch (u8 or i16 pixels), or int32/float coefficients
  const void* in;
  long long in_pitch, in_bstride;    // elements
  int width, height;                 // original (unpadded) size
  int nbx, nby;                      // blocks per row / column (padded size / N)
  long long blocks_per_img;
  int ctas_per_img;
  int in_vec;                        // 1: rows 16-byte aligned, vector loads allowed
  // reconstruction output (float pixels)
  float* out;
  long long out_pitch, out_bstride;  // elements
  int out_vec;
  // coefficient buffer [img][by][bx][N][N] (forward output / inverse input)
  void* coeff;
  // zonal retention
  int r;
  void* kept;                        // [img][blocks][r] in zig-zag order, or null
  unsigned long long slab_mask[16];  // bit (k*N + i): keep row i of slab column k
  // error reduction
  double* partial;                   // one double per CTA, or null
  float scale;                       // integer result -> pixel units (power of two)
};

// Arguments of the per-image SSE -> PSNR finalisation.
struct FinalArgs {
  const double* partial;
  int parts_per_img;
  long long npix;
  double* psnr;                      // [batch], device
  double* sse;                       // [batch], device, or null
};

// Kernel launchers (defined in the per-N translation units).
typedef int (*launch_fn)(const BlockArgs&, int batch, void* stream);

struct KernelSet {
  launch_fn fused;     // forward -> zonal -> inverse (+ SSE partials)
  launch_fn forward;   // forward only -> coefficients
  launch_fn inverse;   // inverse only from coefficients
};

// variant: 0 exact, 1 tilde, 2 hat; conv: 0 paper, 1 transpose; dtype: 0 u8, 1 i16
KernelSet kernels_n8(int variant, int conv, int dtype);
KernelSet kernels_n16(int variant, int conv, int dtype);
KernelSet kernels_n32(int variant, int conv, int dtype);
KernelSet kernels_exact8(int dtype);

// Launch arguments of the persistent pipelined fused kernel.
struct PipeArgs {
  BlockArgs b;
  int units_per_row;       // segments of up to 128/P blocks per block row
  long long units_per_img;
  long long total_units;
  int* err;                // device error word (bit 0: a bulk copy never landed)
  long long wait_limit;    // SM cycles before a stage wait gives up
};

int pipe_launch_n8(int variant, int conv, int dtype, const PipeArgs& pa, int r, int num_sms, void* stream);
int pipe_launch_n16(int variant, int conv, int dtype, const PipeArgs& pa, int r, int num_sms, void* stream);
int pipe_launch_n32(int variant, int conv, int dtype, const PipeArgs& pa, int r, int num_sms, void* stream);

int launch_finalize(const FinalArgs& a, int batch, void* stream);
int launch_zonal(int n, int exact, int conv, const float* s, int r, void* coeff, long long nblocks,
                 float* scaled, void* kept, void* stream);
int launch_psnr_partials(const void* ref, int dtype, long long ref_pitch, long long ref_bstride,
                         const float* recon, long long rec_pitch, long long rec_bstride,
                         int width, int height, int batch, double* partial, int parts_per_img,
                         void* stream);
int psnr_parts_per_img(int height);

// Zig-zag position of (i, j) in an n x n block (anti-diagonals in order;
// row index falling on even diagonals, rising on odd ones).
__host__ __device__ constexpr int zigzag_pos(int n, int i, int j) {
  const int d = i + j;
  if (d < n) {
    const int start = d * (d + 1) / 2;
    return start + ((d & 1) ? i : j);
  }
  const int m = 2 * n - 1 - d;                 // length of diagonal d
  const int start = n * n - m * (m + 1) / 2;
  return start + ((d & 1) ? i - (d - n + 1) : (n - 1) - i);
}

}  // namespace cdct
