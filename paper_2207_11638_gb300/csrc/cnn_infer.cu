// Inference of the CNN size selector: one fused persistent kernel.
//
// The selector proposes, per 32 x 32 region and quantiser slot, one of the 17
// quadtrees of the rate-distortion search (rd.cu) instead of trying them all.
// The paper has no such network: its codec experiment (Sec. 6.2) leaves the
// size choice to the encoder; this kernel is one such choice.
//
// One CTA of 8 warps per SM holds every convolution weight in shared memory
// for its lifetime.  Each warp runs the convolutional trunk of two regions
// at a time entirely in shared memory and registers:
//   conv1 (1 -> 16): implicit GEMM M = 1024 px, N = 16, K = 9 taps (padded to
//                    16); A fragments gathered from the staged region
//   conv2 (16 -> 32): M = 256, N = 32, K = 9 taps x 16 channels
//   conv3 (32 -> 32): M = 64,  N = 32, K = 9 taps x 32 channels
// all as bfloat16 mma.sync m16n8k16 with float32 accumulators; bias, ReLU
// and the 2 x 2 max pool run on the accumulators (the horizontal neighbour
// of a pixel sits 4 lanes away), and each pooled map is written once, as
// bfloat16, into a zero-bordered channel-planar buffer that the next layer
// reads with conflict-free ldmatrix.  The 16 regions of a CTA then share
// one FC1 GEMM (64 x 512 by 512 x 16, Wf1 fragments read from L2/L1 in
// fragment order), and the per-slot head (ReLU, FC2, argmax) runs on CUDA
// cores.  Only the region's pixels are read from HBM and only labels (and
// optional logits / margins) are written.
#include <cuda_runtime.h>

#include <cstdint>

#include "cnn.cuh"
#include "mma.cuh"
#include "common.cuh"
#include "ptx.cuh"

namespace cdct {
namespace {

using namespace cnn;

constexpr int kWarpsI = 8;
constexpr int kThreadsI = 32 * kWarpsI;
constexpr int kGroup = 2 * kWarpsI;             // regions per CTA iteration
constexpr int kFeatPitch = 520;                 // bf16 per feature row (512 + 8)
constexpr int kAct1Bytes = 2 * 18 * 18 * 16;    // [2 planes][18][18][8 ch] bf16
constexpr int kBuf2Bytes = 4 * 10 * 10 * 16;    // act2 [4 planes][10][10][8 ch] bf16, or the staged region
constexpr int kWarpBytes = kAct1Bytes + kBuf2Bytes;
constexpr int kF2Pitch = kHidden + 1;            // Wf2 row pitch in shared memory (floats)
constexpr int kHeadOff = static_cast<int>(kPkConvEnd);
constexpr int kHeadBytes = ((kHidden + kHidden * kSlots + kLabels * kF2Pitch + kLabels) * 4 + 15) / 16 * 16;
constexpr int kWarpOff = kHeadOff + kHeadBytes;
constexpr int kFeatOff = kWarpOff + kWarpsI * kWarpBytes;
constexpr int kUOff = kFeatOff + kGroup * kFeatPitch * 2;
constexpr int kLogitOff = kUOff + kGroup * kHidden * 4;
constexpr int kSmemI = kLogitOff + kGroup * kSlots * kLabels * 4;
static_assert(kWarpOff % 16 == 0 && kFeatOff % 16 == 0 && kUOff % 16 == 0, "alignment");
static_assert(34 * 34 * 2 <= kBuf2Bytes, "staged region fits the act2 buffer");

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

// stage region `reg` (edge-replicated beyond the image) as bf16(x / 64) with a zero border: [34][34]
template <typename InT>
__device__ __forceinline__ void stage_region(const InferArgs& a, long long reg, uint16_t* in0, int lane) {
  const int img = static_cast<int>(reg / a.tiles_per_img);
  const int t = static_cast<int>(reg - static_cast<long long>(img) * a.tiles_per_img);
  const int ty = t / a.tiles_x, tx = t - ty * a.tiles_x;
  const int y0 = ty * 32, x0 = tx * 32;
  const int vrows = min(32, a.height - y0), vcols = min(32, a.width - x0);
  const InT* src = static_cast<const InT*>(a.in) + img * a.bstride;
  const int gx = x0 + min(lane, vcols - 1);
#pragma unroll 8
  for (int r = 0; r < 32; ++r) {
    const int gy = y0 + min(r, vrows - 1);
    const float v = static_cast<float>(src[gy * a.pitch + gx]) * 0.015625f;   // exact in bfloat16
    in0[(r + 1) * 34 + lane + 1] = bf16_bits(v);
  }
  for (int i = lane; i < 34; i += 32) {
    in0[i] = 0;
    in0[33 * 34 + i] = 0;
  }
  in0[(lane + 1) * 34] = 0;
  in0[(lane + 1) * 34 + 33] = 0;
}

// conv1 + bias + ReLU + pool -> act1 (planes of 8 channels, 18 x 18 with a zero border)
__device__ __forceinline__ void conv1_layer(const uint16_t* in0, unsigned char* act1, const uint32_t (&bw)[2][2],
                                            const float* cb, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const int k0 = 2 * t, k1 = 2 * t + 1;
  const int o0 = (k0 / 3) * 34 + k0 % 3, o1 = (k1 / 3) * 34 + k1 % 3;   // taps k < 8 always
  const bool has8 = (t == 0);                                       // tap 8 = (2, 2)
  float bias[2][2];
#pragma unroll
  for (int nt = 0; nt < 2; ++nt) {
    bias[nt][0] = cb[nt * 8 + 2 * t];
    bias[nt][1] = cb[nt * 8 + 2 * t + 1];
  }
#pragma unroll 1
  for (int yp = 0; yp < 16; ++yp) {
#pragma unroll
    for (int xh = 0; xh < 2; ++xh) {
      float acc[2][2][4];
#pragma unroll
      for (int dr = 0; dr < 2; ++dr) {
        const int p0 = (2 * yp + dr) * 34 + xh * 16 + g, p1 = p0 + 8;
        uint32_t af[4];
        af[0] = static_cast<uint32_t>(in0[p0 + o0]) | (static_cast<uint32_t>(in0[p0 + o1]) << 16);
        af[1] = static_cast<uint32_t>(in0[p1 + o0]) | (static_cast<uint32_t>(in0[p1 + o1]) << 16);
        af[2] = has8 ? static_cast<uint32_t>(in0[p0 + 2 * 34 + 2]) : 0u;
        af[3] = has8 ? static_cast<uint32_t>(in0[p1 + 2 * 34 + 2]) : 0u;
#pragma unroll
        for (int nt = 0; nt < 2; ++nt) {
#pragma unroll
          for (int i = 0; i < 4; ++i) acc[dr][nt][i] = 0.f;
          mma_bf16(acc[dr][nt], af, bw[nt]);
        }
      }
#pragma unroll
      for (int nt = 0; nt < 2; ++nt) {
        float v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float b = bias[nt][i & 1];
          v[i] = fmaxf(relu(acc[0][nt][i] + b), relu(acc[1][nt][i] + b));
          v[i] = fmaxf(v[i], __shfl_xor_sync(0xffffffffu, v[i], 4));
        }
        if ((g & 1) == 0) {
          const int px0 = (xh * 16 + g) >> 1, px1 = px0 + 4;
          unsigned char* row = act1 + ((nt * 18 + yp + 1) * 18) * 16 + 4 * t;
          *reinterpret_cast<uint32_t*>(row + (px0 + 1) * 16) = pack_bf16(v[0], v[1]);
          *reinterpret_cast<uint32_t*>(row + (px1 + 1) * 16) = pack_bf16(v[2], v[3]);
        }
      }
    }
  }
}

// conv2 + bias + ReLU + pool: act1 (16 x 16 x 16) -> act2 (8 x 8 x 32, planes of 8, 10 x 10 with a zero border)
__device__ __forceinline__ void conv2_layer(uint32_t act1_s, unsigned char* act2, uint32_t w2_s, const float* cb,
                                            int lane) {
  const int g = lane >> 2, t = lane & 3;
  const uint32_t a_lane = act1_s + (((lane >> 4) * 18 * 18) + (lane & 7) + ((lane >> 3) & 1) * 8) * 16;
  const uint32_t b_lane = w2_s + (((lane & 7) + (lane >> 4) * 8) * kW2Pitch + ((lane >> 3) & 1) * 8) * 2;
  float bias[4][2];
#pragma unroll
  for (int nt = 0; nt < 4; ++nt) {
    bias[nt][0] = cb[16 + nt * 8 + 2 * t];
    bias[nt][1] = cb[16 + nt * 8 + 2 * t + 1];
  }
#pragma unroll 1
  for (int yg = 0; yg < 4; ++yg) {
    float acc[4][4][4];
#pragma unroll
    for (int r = 0; r < 4; ++r)
#pragma unroll
      for (int nt = 0; nt < 4; ++nt)
#pragma unroll
        for (int i = 0; i < 4; ++i) acc[r][nt][i] = 0.f;
#pragma unroll
    for (int tap = 0; tap < 9; ++tap) {
      const int dy = tap / 3, dx = tap % 3;
      uint32_t bf[2][4];
      ldsm_x4(bf[0], b_lane + tap * 32);
      ldsm_x4(bf[1], b_lane + 16 * kW2Pitch * 2 + tap * 32);
#pragma unroll
      for (int r = 0; r < 4; ++r) {
        uint32_t af[4];
        ldsm_x4(af, a_lane + ((4 * yg + r + dy) * 18 + dx) * 16);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const uint32_t b[2] = {bf[nt >> 1][(nt & 1) * 2], bf[nt >> 1][(nt & 1) * 2 + 1]};
          mma_bf16(acc[r][nt], af, b);
        }
      }
    }
#pragma unroll
    for (int rp = 0; rp < 2; ++rp) {
      const int py = 2 * yg + rp;
#pragma unroll
      for (int nt = 0; nt < 4; ++nt) {
        float v[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) {
          const float b = bias[nt][i & 1];
          v[i] = fmaxf(relu(acc[2 * rp][nt][i] + b), relu(acc[2 * rp + 1][nt][i] + b));
          v[i] = fmaxf(v[i], __shfl_xor_sync(0xffffffffu, v[i], 4));
        }
        if ((g & 1) == 0) {
          const int px0 = g >> 1, px1 = px0 + 4;
          unsigned char* row = act2 + ((nt * 10 + py + 1) * 10) * 16 + 4 * t;
          *reinterpret_cast<uint32_t*>(row + (px0 + 1) * 16) = pack_bf16(v[0], v[1]);
          *reinterpret_cast<uint32_t*>(row + (px1 + 1) * 16) = pack_bf16(v[2], v[3]);
        }
      }
    }
  }
}

// conv3 + bias + ReLU + pool: act2 (8 x 8 x 32) -> 512 features (y, x, c) as bf16
__device__ __forceinline__ void conv3_layer(uint32_t act2_s, unsigned char* feat_row, uint32_t w3_s,
                                            const float* cb, int lane) {
  const int g = lane >> 2, t = lane & 3;
  const uint32_t a_lane = act2_s + ((((lane >> 4) * 10 + ((lane >> 3) & 1)) * 10) + (lane & 7)) * 16;
  const uint32_t b_lane = w3_s + (((lane & 7) + (lane >> 4) * 8) * kW3Pitch + ((lane >> 3) & 1) * 8) * 2;
  float acc[4][4][4];
#pragma unroll
  for (int m = 0; m < 4; ++m)
#pragma unroll
    for (int nt = 0; nt < 4; ++nt)
#pragma unroll
      for (int i = 0; i < 4; ++i) acc[m][nt][i] = 0.f;
#pragma unroll 1
  for (int tap = 0; tap < 9; ++tap) {
    const int dy = tap / 3, dx = tap % 3;
#pragma unroll
    for (int c = 0; c < 2; ++c) {
      uint32_t bf[2][4];
      ldsm_x4(bf[0], b_lane + (tap * 32 + c * 16) * 2);
      ldsm_x4(bf[1], b_lane + 16 * kW3Pitch * 2 + (tap * 32 + c * 16) * 2);
#pragma unroll
      for (int m = 0; m < 4; ++m) {
        uint32_t af[4];
        ldsm_x4(af, a_lane + (((2 * c) * 10 + 2 * m + dy) * 10 + dx) * 16);
#pragma unroll
        for (int nt = 0; nt < 4; ++nt) {
          const uint32_t b[2] = {bf[nt >> 1][(nt & 1) * 2], bf[nt >> 1][(nt & 1) * 2 + 1]};
          mma_bf16(acc[m][nt], af, b);
        }
      }
    }
  }
#pragma unroll
  for (int m = 0; m < 4; ++m) {
#pragma unroll
    for (int nt = 0; nt < 4; ++nt) {
      const float b0 = cb[48 + nt * 8 + 2 * t], b1 = cb[48 + nt * 8 + 2 * t + 1];
      float v0 = fmaxf(relu(acc[m][nt][0] + b0), relu(acc[m][nt][2] + b0));
      float v1 = fmaxf(relu(acc[m][nt][1] + b1), relu(acc[m][nt][3] + b1));
      v0 = fmaxf(v0, __shfl_xor_sync(0xffffffffu, v0, 4));
      v1 = fmaxf(v1, __shfl_xor_sync(0xffffffffu, v1, 4));
      if ((g & 1) == 0) {
        const int px = g >> 1;
        *reinterpret_cast<uint32_t*>(feat_row + ((m * 4 + px) * 32 + nt * 8 + 2 * t) * 2) = pack_bf16(v0, v1);
      }
    }
  }
}

template <typename InT>
__global__ void __launch_bounds__(kThreadsI, 1) cnn_infer_kernel(const InferArgs a) {
  extern __shared__ __align__(16) unsigned char sm[];
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int g = lane >> 2, t = lane & 3;
  {
    const uint4* src = reinterpret_cast<const uint4*>(a.packed);
    uint4* dst = reinterpret_cast<uint4*>(sm);
    for (int i = tid; i < static_cast<int>(kPkConvEnd / 16); i += kThreadsI) dst[i] = src[i];
    // head: fb1, Wq as packed; Wf2 rows padded to 65 floats (the logit loop reads
    // one row per label across the lanes); fb2
    const float* hs = reinterpret_cast<const float*>(a.packed + kPkHead);
    float* hd = reinterpret_cast<float*>(sm + kHeadOff);
    constexpr int nq = kHidden + kHidden * kSlots;
    for (int i = tid; i < nq; i += kThreadsI) hd[i] = hs[i];
    for (int i = tid; i < kLabels * kHidden; i += kThreadsI) hd[nq + (i / kHidden) * kF2Pitch + i % kHidden] = hs[nq + i];
    for (int i = tid; i < kLabels; i += kThreadsI) hd[nq + kLabels * kF2Pitch + i] = hs[nq + kLabels * kHidden + i];
  }
  unsigned char* act1 = sm + kWarpOff + warp * kWarpBytes;
  unsigned char* buf2 = act1 + kAct1Bytes;
  for (int i = lane; i < kAct1Bytes / 16; i += 32) reinterpret_cast<uint4*>(act1)[i] = make_uint4(0, 0, 0, 0);
  __syncthreads();

  const float* cb = reinterpret_cast<const float*>(sm + kPkCB);
  uint32_t bw1[2][2];
  {
    const uint16_t* w1 = reinterpret_cast<const uint16_t*>(sm + kPkW1);
#pragma unroll
    for (int nt = 0; nt < 2; ++nt) {
      const uint16_t* row = w1 + (nt * 8 + g) * kW1Pitch;
      bw1[nt][0] = static_cast<uint32_t>(row[2 * t]) | (static_cast<uint32_t>(row[2 * t + 1]) << 16);
      bw1[nt][1] = static_cast<uint32_t>(row[2 * t + 8]) | (static_cast<uint32_t>(row[2 * t + 9]) << 16);
    }
  }
  const uint32_t act1_s = smem_u32(act1), buf2_s = smem_u32(buf2);
  const uint32_t w2_s = smem_u32(sm + kPkW2), w3_s = smem_u32(sm + kPkW3);
  unsigned char* feat = sm + kFeatOff;
  float* u_s = reinterpret_cast<float*>(sm + kUOff);
  float* logit_s = reinterpret_cast<float*>(sm + kLogitOff);
  const float* fb1 = reinterpret_cast<const float*>(sm + kHeadOff);
  const float* wq = fb1 + kHidden;               // [64][4]
  const float* wf2 = wq + kHidden * kSlots;      // [17][65]
  const float* fb2 = wf2 + kLabels * kF2Pitch;   // [17]
  const int ns = a.n_slots;

  for (long long base = static_cast<long long>(blockIdx.x) * kGroup; base < a.n_regions;
       base += static_cast<long long>(gridDim.x) * kGroup) {
#pragma unroll 1
    for (int s = 0; s < 2; ++s) {
      const int slot_row = warp * 2 + s;
      const long long reg = base + slot_row;
      if (reg < a.n_regions) {
        stage_region<InT>(a, reg, reinterpret_cast<uint16_t*>(buf2), lane);
        __syncwarp();
        conv1_layer(reinterpret_cast<const uint16_t*>(buf2), act1, bw1, cb, lane);
        __syncwarp();
        for (int i = lane; i < kBuf2Bytes / 16; i += 32) reinterpret_cast<uint4*>(buf2)[i] = make_uint4(0, 0, 0, 0);
        __syncwarp();
        conv2_layer(act1_s, buf2, w2_s, cb, lane);
        __syncwarp();
        conv3_layer(buf2_s, feat + slot_row * kFeatPitch * 2, w3_s, cb, lane);
        __syncwarp();
      }
    }
    __syncthreads();
    // FC1: u[16 regions][64] = features x Wf1^T; warp = (neuron tile, region tile)
    {
      const int mt = warp & 3, nt = warp >> 2;
      float acc[4] = {0.f, 0.f, 0.f, 0.f};
      const uint4* f1 = reinterpret_cast<const uint4*>(a.packed + kPkF1) + mt * 32 * 32 + lane;
      const uint32_t b_lane = smem_u32(feat) + ((nt * 8 + (lane & 7)) * kFeatPitch + (lane >> 3) * 8) * 2;
#pragma unroll 4
      for (int ks = 0; ks < 32; ks += 2) {
        uint32_t bb[4];
        ldsm_x4(bb, b_lane + ks * 32);
        const uint4 a0 = __ldg(f1 + ks * 32), a1 = __ldg(f1 + (ks + 1) * 32);
        const uint32_t af0[4] = {a0.x, a0.y, a0.z, a0.w}, af1[4] = {a1.x, a1.y, a1.z, a1.w};
        const uint32_t b0[2] = {bb[0], bb[1]}, b1[2] = {bb[2], bb[3]};
        mma_bf16(acc, af0, b0);
        mma_bf16(acc, af1, b1);
      }
      const int n0 = mt * 16 + g, r0 = nt * 8 + 2 * t;
      u_s[r0 * kHidden + n0] = acc[0];
      u_s[(r0 + 1) * kHidden + n0] = acc[1];
      u_s[r0 * kHidden + n0 + 8] = acc[2];
      u_s[(r0 + 1) * kHidden + n0 + 8] = acc[3];
    }
    __syncthreads();
    // head: logits[region][slot][label] = fb2 + Wf2 bf16(relu(u + fb1 + Wq[:, slot]))
    {
      const int per = ns * kLabels;
      for (int task = tid; task < kGroup * per; task += kThreadsI) {
        const int region = task / per, rem = task - region * per;
        const int si = rem / kLabels, j = rem - si * kLabels;
        const int slot = a.slots[si];
        const float* ur = u_s + region * kHidden;
        const float* w = wf2 + j * kF2Pitch;
        float acc = fb2[j];
#pragma unroll 8
        for (int h = 0; h < kHidden; ++h) {
          const float gv = round_bf16(relu((ur[h] + fb1[h]) + wq[h * kSlots + slot]));
          acc = fmaf(w[h], gv, acc);
        }
        logit_s[(region * kSlots + si) * kLabels + j] = acc;
      }
    }
    __syncthreads();
    if (tid < kGroup * ns) {
      const int region = tid / ns, si = tid - region * ns;
      const long long reg = base + region;
      if (reg < a.n_regions) {
        const float* l = logit_s + (region * kSlots + si) * kLabels;
        int best = 0;
        float b1 = l[0], b2 = -INFINITY;
        for (int j = 1; j < kLabels; ++j) {
          if (l[j] > b1) { b2 = b1; b1 = l[j]; best = j; }
          else if (l[j] > b2) b2 = l[j];
        }
        const long long o = static_cast<long long>(si) * a.n_regions + reg;
        a.labels[o] = static_cast<unsigned char>(best);
        if (a.margin != nullptr) a.margin[o] = b1 - b2;
        if (a.logits != nullptr)
          for (int j = 0; j < kLabels; ++j) a.logits[o * kLabels + j] = l[j];
      }
    }
  }
}

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

template <typename InT>
int launch_infer_t(const InferArgs& a, int num_sms, void* stream) {
  auto kern = cnn_infer_kernel<InT>;
  cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, kSmemI);
  if (e != cudaSuccess) return static_cast<int>(e);
  const long long groups = (a.n_regions + kGroup - 1) / kGroup;
  const int grid = static_cast<int>(groups < num_sms ? groups : num_sms);
  if (grid <= 0) return 0;
  kern<<<grid, kThreadsI, kSmemI, static_cast<cudaStream_t>(stream)>>>(a);
  return static_cast<int>(cudaGetLastError());
}

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
                     float* margin, int num_sms, void* stream) {
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
  return dtype == 0 ? launch_infer_t<uint8_t>(a, num_sms, stream) : launch_infer_t<int16_t>(a, num_sms, stream);
}

}  // namespace cdct
