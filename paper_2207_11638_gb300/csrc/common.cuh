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
  int out_v8;                        // 1: rows 32-byte aligned, 256-bit stores allowed
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

// Divisor with its reciprocal for division by multiply-high (see fdiv).
struct FastDiv {
  uint32_t d, m;
};
inline FastDiv make_fastdiv(uint32_t d) {
  FastDiv f;
  f.d = d;
  f.m = static_cast<uint32_t>(0xFFFFFFFFull / d);
  return f;
}

// One image of a descriptor-table batch (same layout as cdct_batch_image).
struct BatchImage {
  const void* data;        // first pixel (device)
  float* recon;            // first reconstructed pixel (device)
  int32_t width, height;
  int64_t pitch, recon_pitch;  // elements
};

// One work unit of a descriptor-table batch, expanded on the host: its
// image's geometry and pointers, its first block row, the segment of that
// row, and the block rows it covers (more than one for a narrow image packed
// `pack_rows` rows per unit).  64 bytes, so that one bulk copy moves it.
struct alignas(16) UnitDesc {
  const void* data;        // first pixel of the image
  float* recon;            // first reconstructed pixel
  int64_t pitch, recon_pitch;
  int32_t width, height, img, by;
  int32_t seg, rows, pad0, pad1;
};

// Launch arguments of the persistent pipelined fused kernel.
struct PipeArgs {
  BlockArgs b;
  int units_per_row;       // segments of up to 128/P blocks per block row
  long long units_per_img;
  long long total_units;   // < 2^31
  FastDiv div_img, div_row;
  const UnitDesc* unit_map;  // descriptor-table batches: one record per work unit (null: uniform batch)
  int* err;                // device error word (bit 0: a bulk copy never landed)
  long long wait_limit;    // SM cycles before a stage wait gives up
  int drop_copies;         // failure-detection test: arm the stage barriers but issue no copy
};

// Failure-detection test hook (cdct_set_fault_injection): the current mode
// bits and the wait limit, in SM cycles, the kernels use while it is set.
constexpr long long kDefaultWaitLimit = 1ll << 31;   // about one second of SM clock
int fault_mode(long long* wait_limit);

// Tuning of the pipelined kernel: staging depth (0 = default for N) and
// resident CTAs per SM used for the grid (0 = as many as fit).
struct PipeTuning {
  int stages;
  int ctas_per_sm;
};
int pipe_launch_n8(int variant, int conv, int dtype, const PipeArgs& pa, int r, int num_sms, PipeTuning t,
                   void* stream);
int pipe_launch_n16(int variant, int conv, int dtype, const PipeArgs& pa, int r, int num_sms, PipeTuning t,
                    void* stream);
int pipe_launch_n32(int variant, int conv, int dtype, const PipeArgs& pa, int r, int num_sms, PipeTuning t,
                    void* stream);

int launch_finalize(const FinalArgs& a, int batch, void* stream);

// Rate-distortion quadtree search (rd.cu)
int rd_table_words();
void rd_tables(int variant, int* out);
// mode 0: search every region; 1: search the listed regions (subset, device count);
// 2: evaluate given labels (in_labels) -> ev_cost / ev_dist / ev_bits
struct RdModeArgs {
  int mode;
  const long long* subset;
  const long long* subset_count;
  long long max_count;
  const unsigned char* in_labels;
  unsigned long long* ev_cost;
  unsigned long long* ev_dist;
  int* ev_bits;
};
int launch_rd(int variant, int dtype, const void* in, long long pitch, long long bstride, int width, int height,
              int batch, const int* host_tables, const int* q, int nq, const unsigned long long* lam_lo,
              const unsigned long long* lam_hi, unsigned char* labels, unsigned long long* part_cost, int num_sms,
              void* stream, const RdModeArgs* mode = nullptr);
// per-image PSNR of a descriptor-table batch (warps_per_unit partials per unit)
int launch_finalize_table(const double* partial, const long long* unit_prefix, const BatchImage* images,
                          int n_images, int warps_per_unit, double* psnr, void* stream);
int launch_zonal(int n, int exact, int conv, const float* s, int r, void* coeff, long long nblocks,
                 float* scaled, void* kept, void* stream);
int launch_psnr_partials(const void* ref, int dtype, long long ref_pitch, long long ref_bstride,
                         const float* recon, long long rec_pitch, long long rec_bstride,
                         int width, int height, int batch, double* partial, int parts_per_img,
                         void* stream);
int psnr_parts_per_img(int height);
// mean SSIM per image (ssim.cu): window-position tiles per image, and the launch
long long ssim_tiles(int width, int height);
int ssim_launch(const void* ref, int dtype, long long ref_pitch, long long ref_bstride, const float* rec,
                long long rec_pitch, long long rec_bstride, int width, int height, int batch, double* partial,
                double* ssim, void* stream);

// Block rows per work unit of a descriptor-table image `nbx` blocks wide (S
// blocks per unit): narrow images (at most half a unit wide) pack whole block
// rows into one unit so that the unit's lanes are not left idle.
__host__ __device__ constexpr int pack_rows(int nbx, int S) { return nbx <= S / 2 ? S / nbx : 1; }

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

// zig-zag cut: 1 + the highest row or column index among the first r
// positions (rows and columns can differ by one: an even partial diagonal
// starts at its bottom-left end, an odd one at its top-right end)
__host__ __device__ constexpr int zonal_extent(int n, int r) {
  int e = 0;
  for (int i = 0; i < n; ++i)
    for (int j = 0; j < n; ++j)
      if (zigzag_pos(n, i, j) < r) {
        if (j + 1 > e) e = j + 1;
        if (i + 1 > e) e = i + 1;
      }
  return e;
}

// Global coefficient row / column of local (i, k) in 8 x 8 sub-block q.
//   N = 16: q = a*2 + b, row = 2i + a, col = 2k + b
//   N = 32: q = hr*8 + ar*4 + c with c = h*2 + a',
//           row = 4i + 2ar + hr, col = 4k + 2a' + h
__host__ __device__ constexpr int sub_row_of(int n, int q, int i) {
  return n == 8 ? i : (n == 16 ? 2 * i + (q >> 1) : 4 * i + 2 * ((q >> 2) & 1) + (q >> 3));
}
__host__ __device__ constexpr int sub_col_of(int n, int q, int k) {
  return n == 8 ? k : (n == 16 ? 2 * k + (q & 1) : 4 * k + 2 * (q & 1) + ((q >> 1) & 1));
}
// bit (k * 8 + i): keep local row i of local column k of sub-block q
__host__ __device__ constexpr unsigned long long sub_mask(int n, int r, int q) {
  unsigned long long m = 0;
  for (int k = 0; k < 8; ++k)
    for (int i = 0; i < 8; ++i)
      if (zigzag_pos(n, sub_row_of(n, q, i), sub_col_of(n, q, k)) < r) m |= 1ull << (k * 8 + i);
  return m;
}
// bits kept in at least one / in every sub-block of an N-point block
__host__ __device__ constexpr unsigned long long sub_mask_any(int n, int r) {
  unsigned long long m = 0;
  for (int q = 0; q < (n / 8) * (n / 8); ++q) m |= sub_mask(n, r, q);
  return m;
}
__host__ __device__ constexpr unsigned long long sub_mask_all(int n, int r) {
  unsigned long long m = ~0ull;
  for (int q = 0; q < (n / 8) * (n / 8); ++q) m &= sub_mask(n, r, q);
  return m;
}

}  // namespace cdct
