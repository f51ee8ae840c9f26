// Layouts shared by the CNN size-selector kernels (cnn_infer.cu, cnn_train.cu).
//
// Network (per 32 x 32 region x, activations NHWC):
//   a0 = x / 64;  a_l = maxpool2(relu(conv3x3_l(a_{l-1}) + b_l)),  l = 1..3, channels 1-16-32-32
//   h = a_3 flattened (y, x, c): 512 features;  u = Wf1 h
//   per quantiser slot k:  g_k = relu(u + bf1 + Wq[:, k]);  logits_k = Wf2 g_k + bf2  (17 labels)
// Weights are used as bfloat16 copies of float32 master weights; activations
// are stored as bfloat16; products accumulate in float32.
#pragma once
#include <cstddef>
#include <cstdint>

namespace cdct {
namespace cnn {

constexpr int kLabels = 17, kHidden = 64, kFeat = 512, kSlots = 4;
constexpr int kC1 = 16, kC2 = 32, kC3 = 32;

// flat float32 parameter vector (offsets in floats)
constexpr int kOffW1 = 0;                        // [16][3][3][1]
constexpr int kOffB1 = kOffW1 + 16 * 9;          // [16]
constexpr int kOffW2 = kOffB1 + 16;              // [32][3][3][16]
constexpr int kOffB2 = kOffW2 + 32 * 9 * 16;     // [32]
constexpr int kOffW3 = kOffB2 + 32;              // [32][3][3][32]
constexpr int kOffB3 = kOffW3 + 32 * 9 * 32;     // [32]
constexpr int kOffF1 = kOffB3 + 32;              // [64][512]
constexpr int kOffQ = kOffF1 + kHidden * kFeat;  // [64][4]
constexpr int kOffFB1 = kOffQ + kHidden * kSlots;  // [64]
constexpr int kOffF2 = kOffFB1 + kHidden;        // [17][64]
constexpr int kOffFB2 = kOffF2 + kLabels * kHidden;  // [17]
constexpr int kParams = kOffFB2 + kLabels;       // 48241

// Packed inference weights (bytes).  Row pitches are padded so that the
// ldmatrix reads of 8 rows touch 32 distinct banks.
constexpr int kW1Pitch = 24;    // bf16 per row: 9 taps, zero to 16, pad to 24
constexpr int kW2Pitch = 152;   // 144 + 8
constexpr int kW3Pitch = 296;   // 288 + 8
constexpr size_t kPkW1 = 0;                                  // [16][24] bf16
constexpr size_t kPkW2 = kPkW1 + 16 * kW1Pitch * 2;          // [32][152] bf16
constexpr size_t kPkW3 = kPkW2 + 32 * kW2Pitch * 2;          // [32][296] bf16
constexpr size_t kPkCB = kPkW3 + 32 * kW3Pitch * 2;          // b1[16] b2[32] b3[32] float
constexpr size_t kPkConvEnd = kPkCB + 80 * 4;                // conv section: copied to shared memory
constexpr size_t kPkF1 = kPkConvEnd;                         // [4 mt][32 ks][32 lane] uint4: A fragments of Wf1
constexpr size_t kPkHead = kPkF1 + 4 * 32 * 32 * 16;         // head section: copied to shared memory
constexpr size_t kPkFB1 = kPkHead;                           // [64] float
constexpr size_t kPkQ = kPkFB1 + kHidden * 4;                // [64][4] float (bfloat16 values)
constexpr size_t kPkF2 = kPkQ + kHidden * kSlots * 4;        // [17][64] float (bfloat16 values)
constexpr size_t kPkFB2 = kPkF2 + kLabels * kHidden * 4;     // [17] float, padded to 20
constexpr size_t kPkHeadEnd = kPkFB2 + 20 * 4;
constexpr size_t kPackedBytes = (kPkHeadEnd + 255) / 256 * 256;

static_assert(kPkW2 % 16 == 0 && kPkW3 % 16 == 0 && kPkCB % 16 == 0 && kPkF1 % 16 == 0 && kPkHead % 16 == 0,
              "packed sections must be 16-byte aligned");
static_assert(kParams == 48241, "parameter count");

}  // namespace cnn

// launchers (cnn_infer.cu)
int cnn_pack_launch(const float* params, void* packed, void* stream);
int cnn_infer_launch(const void* packed, const void* in, int dtype, long long pitch, long long bstride, int width,
                     int height, int batch, const int* slots, int n_slots, unsigned char* labels, float* logits,
                     float* margin, int num_sms, int* err, void* stream);
int cnn_select_launch(const float* margin, long long n, int ns, float threshold, long long* idx, long long* count,
                      int num_sms, void* stream);
// launchers (cnn_train.cu)
size_t cnn_train_workspace(long long batch);
int cnn_grad_launch(const float* params, const int16_t* regions, int B, const int* slots, int ns,
                    const unsigned char* labels, const unsigned long long* pcost, float mu, float* grad,
                    float* loss, void* workspace, int* err, void* stream);
int cnn_adam_launch(float* params, const float* grad, float* m, float* v, int step, float lr, float beta1,
                    float beta2, float eps, void* stream);

}  // namespace cdct
