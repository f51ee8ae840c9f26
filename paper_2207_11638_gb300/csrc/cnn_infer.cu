// Inference of the CNN size selector: one fused persistent kernel.
//
// The selector proposes, per 32 x 32 region and quantiser slot, one of the 17
// quadtrees of the rate-distortion search (rd.cu) instead of trying them all.
// The paper has no such network: its codec experiment (Sec. 6.2) leaves the
// size choice to the encoder; this kernel is one such choice.
//
// The kernel (cnn_infer_tc.cuh) runs the convolutional trunk on the tensor
// cores (tcgen05, accumulators in tensor memory), tiled by pooling windows so
// that the 2 x 2 max pool stays in registers; 16 regions per CTA share one
// FC1 GEMM (64 x 512 by 512 x 16, Wf1 fragments read from L2/L1 in fragment
// order, warp-level MMA), and the per-slot head (ReLU, FC2, argmax) runs on
// CUDA cores.  Only the region's pixels are read from HBM and only labels
// (and optional logits / margins) are written.
#include <cuda_runtime.h>

#include <cstdint>

#include "cnn.cuh"
#include "mma.cuh"
#include "common.cuh"
#include "ptx.cuh"
#include "tcgen05.cuh"

namespace cdct {
namespace {

using namespace cnn;

constexpr int kFeatPitch = 520;                 // bf16 per feature row (512 + 8)
constexpr int kF2Pitch = kHidden + 4;            // Wf2 row pitch in shared memory (floats; 16-byte rows)
constexpr int kHeadBytes = ((kHidden + kHidden * kSlots + kLabels * kF2Pitch + kLabels) * 4 + 15) / 16 * 16;

struct InferArgs {
  const unsigned char* packed;
  const void* in;
  long long pitch, bstride;
  int width, height, tiles_x, tiles_per_img;
  long long n_regions;
  int n_slots;
  int slots[kSlots];
  unsigned char* labels;   // [n_slots][n_regions]
  float* logits;           // [n_slots][n_regions][17] or null
  float* margin;           // [n_slots][n_regions] or null
};

__device__ __forceinline__ float relu(float x) { return fmaxf(x, 0.f); }

// params (float32, flat) -> packed inference weights (see cnn.cuh)
__global__ void cnn_pack_kernel(const float* __restrict__ p, unsigned char* __restrict__ out) {
  constexpr int n1 = 16 * kW1Pitch, n2 = 32 * kW2Pitch, n3 = 32 * kW3Pitch, ncb = 80, nf1 = 4 * 32 * 32 * 8;
  constexpr int nfb1 = kHidden, nq = kHidden * kSlots, nf2 = kLabels * kHidden, nfb2 = 20;
  constexpr int total = n1 + n2 + n3 + ncb + nf1 + nfb1 + nq + nf2 + nfb2;
  for (int i = blockIdx.x * blockDim.x + threadIdx.x; i < total; i += gridDim.x * blockDim.x) {
    int k = i;
    if (k < n1) {
      const int row = k / kW1Pitch, c = k % kW1Pitch;
      reinterpret_cast<uint16_t*>(out + kPkW1)[k] = bf16_bits(c < 9 ? p[kOffW1 + row * 9 + c] : 0.f);
      continue;
    }
    k -= n1;
    if (k < n2) {
      const int row = k / kW2Pitch, c = k % kW2Pitch;
      reinterpret_cast<uint16_t*>(out + kPkW2)[k] = bf16_bits(c < 144 ? p[kOffW2 + row * 144 + c] : 0.f);
      continue;
    }
    k -= n2;
    if (k < n3) {
      const int row = k / kW3Pitch, c = k % kW3Pitch;
      reinterpret_cast<uint16_t*>(out + kPkW3)[k] = bf16_bits(c < 288 ? p[kOffW3 + row * 288 + c] : 0.f);
      continue;
    }
    k -= n3;
    if (k < ncb) {
      reinterpret_cast<float*>(out + kPkCB)[k] =
          k < 16 ? p[kOffB1 + k] : (k < 48 ? p[kOffB2 + k - 16] : p[kOffB3 + k - 48]);
      continue;
    }
    k -= ncb;
    if (k < nf1) {
      const int e = k & 7, lane = (k >> 3) & 31, ks = (k >> 8) & 31, mt = k >> 13;
      const int r = e >> 1, hi = e & 1;
      const int row = mt * 16 + (lane >> 2) + ((r & 1) ? 8 : 0);
      const int col = ks * 16 + 2 * (lane & 3) + ((r & 2) ? 8 : 0) + hi;
      reinterpret_cast<uint16_t*>(out + kPkF1)[k] = bf16_bits(p[kOffF1 + row * kFeat + col]);
      continue;
    }
    k -= nf1;
    if (k < nfb1) { reinterpret_cast<float*>(out + kPkFB1)[k] = p[kOffFB1 + k]; continue; }
    k -= nfb1;
    if (k < nq) { reinterpret_cast<float*>(out + kPkQ)[k] = round_bf16(p[kOffQ + k]); continue; }
    k -= nq;
    if (k < nf2) { reinterpret_cast<float*>(out + kPkF2)[k] = round_bf16(p[kOffF2 + k]); continue; }
    k -= nf2;
    reinterpret_cast<float*>(out + kPkFB2)[k] = k < kLabels ? p[kOffFB2 + k] : 0.f;
  }
}

// regions whose smallest margin over the slots is below `threshold`: their
// numbers go to idx[0 .. *count) (in no particular order)
__global__ void select_kernel(const float* __restrict__ margin, long long n, int ns, float threshold,
                              long long* __restrict__ idx, unsigned long long* __restrict__ count) {
  for (long long r = static_cast<long long>(blockIdx.x) * blockDim.x + threadIdx.x; r < n;
       r += static_cast<long long>(gridDim.x) * blockDim.x) {
    float m = margin[r];
    for (int si = 1; si < ns; ++si) m = fminf(m, margin[static_cast<long long>(si) * n + r]);
    if (m < threshold) idx[atomicAdd(count, 1ull)] = r;
  }
}

#include "cnn_infer_tc.cuh"

}  // namespace

int cnn_select_launch(const float* margin, long long n, int ns, float threshold, long long* idx, long long* count,
                      int num_sms, void* stream) {
  cudaStream_t st = static_cast<cudaStream_t>(stream);
  cudaError_t e = cudaMemsetAsync(count, 0, sizeof(long long), st);
  if (e != cudaSuccess) return static_cast<int>(e);
  const long long blocks = (n + 255) / 256;
  const int grid = static_cast<int>(blocks < 4LL * num_sms ? blocks : 4LL * num_sms);
  if (grid <= 0) return 0;
  select_kernel<<<grid, 256, 0, st>>>(margin, n, ns, threshold, idx, reinterpret_cast<unsigned long long*>(count));
  return static_cast<int>(cudaGetLastError());
}

int cnn_pack_launch(const float* params, void* packed, void* stream) {
  cnn_pack_kernel<<<64, 256, 0, static_cast<cudaStream_t>(stream)>>>(params, static_cast<unsigned char*>(packed));
  return static_cast<int>(cudaGetLastError());
}

int cnn_infer_launch(const void* packed, const void* in, int dtype, long long pitch, long long bstride, int width,
                     int height, int batch, const int* slots, int n_slots, unsigned char* labels, float* logits,
                     float* margin, int num_sms, int* err, void* stream) {
  InferArgs a;
  a.packed = static_cast<const unsigned char*>(packed);
  a.in = in;
  a.pitch = pitch;
  a.bstride = bstride;
  a.width = width;
  a.height = height;
  a.tiles_x = (width + 31) / 32;
  a.tiles_per_img = a.tiles_x * ((height + 31) / 32);
  a.n_regions = static_cast<long long>(batch) * a.tiles_per_img;
  a.n_slots = n_slots;
  for (int k = 0; k < kSlots; ++k) a.slots[k] = k < n_slots ? slots[k] : 0;
  a.labels = labels;
  a.logits = logits;
  a.margin = margin;
  return dtype == 0 ? launch_infer_tc_t<uint8_t>(a, num_sms, err, stream) : launch_infer_tc_t<int16_t>(a, num_sms, err, stream);
}

}  // namespace cdct
