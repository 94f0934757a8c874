// mlp.cu — the learned proposal network: MLP 6 -> 64 -> 64 -> 256 (GELU),
// BF16 weights, FP32 accumulation, trained on the GPU with these kernels.
//
// Input of a ray: its origin mapped to the scene box ([-1, 1]^3, with box
// centre c and half extents h: (o - c) / h) and its direction.  Output: 256
// logits, one per depth-8 subtree of the BVH (the "frontier").
//
// Parameter layout (floats, the same for the FP32 master copy, the BF16
// copy, the gradient and both Adam moments):
//   W1[64][6] @0, b1[64] @384, W2[64][64] @448, b2[64] @4544,
//   W3[256][64] @4608, b3[256] @20992;  P = 21248.
//
// Training step (sc_mlp_grad, then sc_mlp_adam): forward over the batch
// storing the pre-activations A1, A2 and dZ = (softmax(z) - onehot(y)) / B
// (the gradient of the mean cross-entropy); weight gradients as split-K
// reductions over the batch; the hidden backward dA = (dZ W) * gelu'(A);
// Adam on the FP32 master copy, then re-rounding to BF16.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include <cmath>
#include <cstring>
#include <mutex>
#include <vector>

#include "host/internal.h"

using namespace sc;

namespace mlpk {

constexpr int IN = 6, H = 64, OUT = 256;
constexpr int OFF_W1 = 0, OFF_B1 = 384, OFF_W2 = 448, OFF_B2 = 4544, OFF_W3 = 4608,
              OFF_B3 = 20992, P = 21248;
constexpr int kThreads = 128;

__device__ __forceinline__ float gelu(float x) {
  return 0.5f * x * (1.0f + erff(x * 0.70710678118654752f));
}
__device__ __forceinline__ float gelu_grad(float x) {
  return 0.5f * (1.0f + erff(x * 0.70710678118654752f)) +
         x * 0.39894228040143268f * expf(-0.5f * x * x);
}

// Input features of one ray.
__device__ __forceinline__ void features(const float4 ra, const float4 rb, const float* box,
                                         float* x) {
  x[0] = (ra.x - box[0]) / box[3];
  x[1] = (ra.y - box[1]) / box[4];
  x[2] = (ra.z - box[2]) / box[5];
  x[3] = rb.x;
  x[4] = rb.y;
  x[5] = rb.z;
}

// Weights staged in shared memory as floats (from the BF16 copy).
struct SmemW {
  float w[P];
};

__device__ __forceinline__ void stage(SmemW& s, const __nv_bfloat16* wb) {
  for (int i = threadIdx.x; i < P; i += blockDim.x) s.w[i] = __bfloat162float(wb[i]);
}

// h1 = gelu(W1 x + b1), h2 = gelu(W2 h1 + b2); the pre-activations are
// written to the rows a1 / a2 when those are not null (training).
__device__ __forceinline__ void hidden(const SmemW& s, const float* x, float* a1, float* h1,
                                       float* a2, float* h2) {
#pragma unroll
  for (int o = 0; o < H; ++o) {
    float acc = s.w[OFF_B1 + o];
#pragma unroll
    for (int i = 0; i < IN; ++i) acc += s.w[OFF_W1 + o * IN + i] * x[i];
    if (a1) a1[o] = acc;
    h1[o] = gelu(acc);
  }
#pragma unroll
  for (int o = 0; o < H; ++o) {
    const float4* row = reinterpret_cast<const float4*>(&s.w[OFF_W2 + o * H]);
    float acc0 = s.w[OFF_B2 + o], acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
#pragma unroll
    for (int i = 0; i < H / 4; ++i) {
      const float4 w = row[i];
      acc0 += w.x * h1[4 * i];
      acc1 += w.y * h1[4 * i + 1];
      acc2 += w.z * h1[4 * i + 2];
      acc3 += w.w * h1[4 * i + 3];
    }
    const float acc = (acc0 + acc1) + (acc2 + acc3);
    if (a2) a2[o] = acc;
    h2[o] = gelu(acc);
  }
}

__device__ __forceinline__ float logit(const SmemW& s, const float* h2, int o) {
  const float4* row = reinterpret_cast<const float4*>(&s.w[OFF_W3 + o * H]);
  float acc0 = s.w[OFF_B3 + o], acc1 = 0.f, acc2 = 0.f, acc3 = 0.f;
#pragma unroll
  for (int i = 0; i < H / 4; ++i) {
    const float4 w = row[i];
    acc0 += w.x * h2[4 * i];
    acc1 += w.y * h2[4 * i + 1];
    acc2 += w.z * h2[4 * i + 2];
    acc3 += w.w * h2[4 * i + 3];
  }
  return (acc0 + acc1) + (acc2 + acc3);
}

// Inference: top-1 class (and optionally all logits) of each ray; -1 when
// the top-1 softmax probability is below min_prob (min_prob <= 0: never).
__global__ void __launch_bounds__(kThreads) infer_kernel(const __nv_bfloat16* wb,
                                                         const float4* rays, long long n,
                                                         const float* box, int* cls,
                                                         float* logits, float min_prob) {
  extern __shared__ float4 smem_raw[];
  SmemW& s = *reinterpret_cast<SmemW*>(smem_raw);
  stage(s, wb);
  __syncthreads();
  float bx[6];
  for (int k = 0; k < 6; ++k) bx[k] = box[k];
  for (long long r = (long long)blockIdx.x * blockDim.x + threadIdx.x; r < n;
       r += (long long)gridDim.x * blockDim.x) {
    float x[IN], h1[H], h2[H];
    features(__ldg(&rays[2 * r]), __ldg(&rays[2 * r + 1]), bx, x);
    hidden(s, x, nullptr, h1, nullptr, h2);
    float best = -INFINITY, se = 0.0f;  // running max and sum of exp(z - max)
    int bi = 0;
    for (int o = 0; o < OUT; ++o) {
      const float z = logit(s, h2, o);
      if (logits) logits[r * OUT + o] = z;
      if (z > best) {
        if (min_prob > 0.0f) se = se * expf(best - z) + 1.0f;
        best = z;
        bi = o;
      } else if (min_prob > 0.0f) {
        se += expf(z - best);
      }
    }
    // top-1 probability = 1 / se
    cls[r] = (min_prob > 0.0f && se * min_prob > 1.0f) ? -1 : bi;
  }
}

// Training forward: A1, A2 and dZ = (softmax - onehot) / B; loss sum.
__global__ void __launch_bounds__(kThreads) train_fwd_kernel(
    const __nv_bfloat16* wb, const float4* rays, const int* labels, long long B,
    const float* box, float* A1, float* A2, float* dZ, float* loss) {
  extern __shared__ float4 smem_raw[];
  SmemW& s = *reinterpret_cast<SmemW*>(smem_raw);
  stage(s, wb);
  __syncthreads();
  float bx[6];
  for (int k = 0; k < 6; ++k) bx[k] = box[k];
  float lsum = 0.0f;
  const float invB = 1.0f / (float)B;
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < B;
       b += (long long)gridDim.x * blockDim.x) {
    float x[IN], h1[H], h2[H];
    features(__ldg(&rays[2 * b]), __ldg(&rays[2 * b + 1]), bx, x);
    hidden(s, x, A1 + b * H, h1, A2 + b * H, h2);
    float* z = dZ + b * OUT;
    float m = -INFINITY;
    for (int o = 0; o < OUT; ++o) {
      const float v = logit(s, h2, o);
      z[o] = v;
      m = fmaxf(m, v);
    }
    float se = 0.0f;
    for (int o = 0; o < OUT; ++o) se += expf(z[o] - m);
    const int y = labels[b];
    lsum += (logf(se) + m) - z[y];
    const float inv = 1.0f / se;
    for (int o = 0; o < OUT; ++o) z[o] = (expf(z[o] - m) * inv - (o == y ? 1.0f : 0.0f)) * invB;
  }
  // block reduction of the loss
  __shared__ float red[kThreads];
  red[threadIdx.x] = lsum;
  __syncthreads();
  for (int st = blockDim.x / 2; st > 0; st >>= 1) {
    if ((int)threadIdx.x < st) red[threadIdx.x] += red[threadIdx.x + st];
    __syncthreads();
  }
  if (threadIdx.x == 0) atomicAdd(loss, red[0] * invB);
}

// dW[o][i] += sum_b dA[b][o] * Hin[b][i] and db[o] += sum_b dA[b][o], where
// Hin = gelu(Asrc) (act = 1), Asrc itself (act = 0) or the ray features
// (act = 2, Asrc = rays).  Split-K over the batch: each block reduces a
// batch slice for a 32 x 32 output tile and adds it atomically.
constexpr int TG = 32, KB = 32;
__global__ void __launch_bounds__(256) grad_w_kernel(const float* dA, int O, const float* Asrc,
                                                     int I, int act, const float* box,
                                                     long long B, long long slice, float* dW,
                                                     float* db) {
  __shared__ float sa[KB][TG + 1];
  __shared__ float sh[KB][TG + 1];
  const int o0 = blockIdx.y * TG, i0 = blockIdx.z * TG;
  const long long b_begin = (long long)blockIdx.x * slice;
  const long long b_end = b_begin + slice < B ? b_begin + slice : B;
  const int tx = threadIdx.x & 31, ty = threadIdx.x >> 5;  // 32 x 8
  float acc[4] = {0.f, 0.f, 0.f, 0.f};
  float accb[4] = {0.f, 0.f, 0.f, 0.f};
  for (long long b0 = b_begin; b0 < b_end; b0 += KB) {
    for (int r = ty; r < KB; r += 8) {
      const long long b = b0 + r;
      const bool ok = b < b_end;
      sa[r][tx] = (ok && o0 + tx < O) ? dA[b * O + o0 + tx] : 0.0f;
      float hv = 0.0f;
      if (ok && i0 + tx < I) {
        if (act == 2) {
          const float4* rr = reinterpret_cast<const float4*>(Asrc) + 2 * b;
          float x[IN];
          features(rr[0], rr[1], box, x);
          hv = x[i0 + tx];
        } else {
          const float a = Asrc[b * I + i0 + tx];
          hv = act ? gelu(a) : a;
        }
      }
      sh[r][tx] = hv;
    }
    __syncthreads();
#pragma unroll 4
    for (int r = 0; r < KB; ++r) {
      const float hv = sh[r][tx];
#pragma unroll
      for (int j = 0; j < 4; ++j) {
        const float av = sa[r][ty + 8 * j];
        acc[j] += av * hv;
        if (blockIdx.z == 0 && tx == 0) accb[j] += av;
      }
    }
    __syncthreads();
  }
#pragma unroll
  for (int j = 0; j < 4; ++j) {
    const int o = o0 + ty + 8 * j, i = i0 + tx;
    if (o < O && i < I) atomicAdd(&dW[o * I + i], acc[j]);
    if (blockIdx.z == 0 && tx == 0 && o < O) atomicAdd(&db[o], accb[j]);
  }
}

// dAprev[b][i] = (sum_o dA[b][o] * W[o][i]) * gelu'(Aprev[b][i]), W from
// the BF16 copy (as used by the forward pass).
template <int O>
__global__ void __launch_bounds__(kThreads) back_hidden_kernel(const float* dA,
                                                              const __nv_bfloat16* wb, int off_w,
                                                              const float* Aprev, long long B,
                                                              float* dAprev) {
  extern __shared__ float4 smem_w4[];
  float* w = reinterpret_cast<float*>(smem_w4);
  for (int k = threadIdx.x; k < O * H; k += blockDim.x) w[k] = __bfloat162float(wb[off_w + k]);
  __syncthreads();
  for (long long b = (long long)blockIdx.x * blockDim.x + threadIdx.x; b < B;
       b += (long long)gridDim.x * blockDim.x) {
    float acc[H];
#pragma unroll
    for (int i = 0; i < H; ++i) acc[i] = 0.0f;
    for (int o = 0; o < O; ++o) {
      const float g = dA[b * O + o];
      const float4* row = reinterpret_cast<const float4*>(&w[o * H]);
#pragma unroll
      for (int i = 0; i < H / 4; ++i) {
        const float4 v = row[i];
        acc[4 * i] += g * v.x;
        acc[4 * i + 1] += g * v.y;
        acc[4 * i + 2] += g * v.z;
        acc[4 * i + 3] += g * v.w;
      }
    }
#pragma unroll
    for (int i = 0; i < H; ++i) dAprev[b * H + i] = acc[i] * gelu_grad(Aprev[b * H + i]);
  }
}

// Adam on the FP32 master copy; refreshes the BF16 copy; zeroes the
// gradient.  bc1 = 1 / (1 - beta1^t), bc2 = 1 / (1 - beta2^t).
__global__ void adam_kernel(float* w, __nv_bfloat16* wb, float* g, float* m, float* v, float lr,
                            float beta1, float beta2, float eps, float bc1, float bc2) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= P) return;
  const float gi = g[i];
  const float mi = beta1 * m[i] + (1.0f - beta1) * gi;
  const float vi = beta2 * v[i] + (1.0f - beta2) * gi * gi;
  m[i] = mi;
  v[i] = vi;
  const float wi = w[i] - lr * (mi * bc1) / (sqrtf(vi * bc2) + eps);
  w[i] = wi;
  wb[i] = __float2bfloat16_rn(wi);
  g[i] = 0.0f;
}

__global__ void to_bf16_kernel(const float* w, __nv_bfloat16* wb) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i < P) wb[i] = __float2bfloat16_rn(w[i]);
}

// Training pairs from a traced wave: rays with a hit and their subtree
// class (class_of_tri[hit id]), appended with a warp-aggregated atomic.
__global__ void labels_kernel(const float4* rays, const float4* hits, long long n,
                              const unsigned char* class_of_tri, float4* out_rays, int* out_lbl,
                              unsigned* count, long long cap) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  int cls = -1;
  if (i < n) {
    const int id = __float_as_int(hits[i].y);
    if (id >= 0) cls = class_of_tri[id];
  }
  const unsigned lane = threadIdx.x & 31u;
  const unsigned m = __ballot_sync(0xffffffffu, cls >= 0);
  if (!m) return;
  const int leader = __ffs(m) - 1;
  unsigned base = 0;
  if ((int)lane == leader) base = atomicAdd(count, (unsigned)__popc(m));
  base = __shfl_sync(0xffffffffu, base, leader);
  if (cls >= 0) {
    const long long pos = (long long)base + __popc(m & ((1u << lane) - 1u));
    if (pos < cap) {
      out_rays[2 * pos] = rays[2 * i];
      out_rays[2 * pos + 1] = rays[2 * i + 1];
      out_lbl[pos] = cls;
    }
  }
}

// Minibatch gather through a pseudo-random permutation of [0, n) (device
// shuffling for training): a 4-round Feistel network on the smallest
// domain of 2h bits that holds n, with cycle walking (Black & Rogaway,
// "Ciphers with arbitrary finite domains", 2002): a value outside [0, n)
// is permuted again until it falls inside, which ends because the walk
// follows the cycle of the start value.
__device__ __forceinline__ uint32_t feistel_round(uint32_t x, uint32_t k) {
  uint32_t v = (x ^ k) * 0x9E3779B1u;
  v ^= v >> 15;
  v *= 0x85EBCA77u;
  v ^= v >> 13;
  return v;
}

__device__ __forceinline__ uint32_t feistel(uint32_t x, int h, const uint32_t* key) {
  const uint32_t mask = (h >= 32) ? 0xFFFFFFFFu : ((1u << h) - 1u);
  uint32_t L = x >> h, R = x & mask;
#pragma unroll
  for (int r = 0; r < 4; ++r) {
    const uint32_t t = R;
    R = (L ^ feistel_round(R, key[r])) & mask;
    L = t;
  }
  return (L << h) | R;
}

__global__ void gather_kernel(const float4* rays, const int* labels, long long n, int h,
                              uint4 key, long long start, long long batch, float4* out_rays,
                              int* out_labels) {
  const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= batch) return;
  const uint32_t k[4] = {key.x, key.y, key.z, key.w};
  uint32_t y = feistel((uint32_t)(start + i), h, k);
  while ((long long)y >= n) y = feistel(y, h, k);
  out_rays[2 * i] = rays[2 * (long long)y];
  out_rays[2 * i + 1] = rays[2 * (long long)y + 1];
  out_labels[i] = labels[y];
}

// ------------------------------------------------ tensor-core inference --
// Layers 2 and 3 of the forward pass on the 5th-generation tensor cores:
// per tile of 128 rays, tcgen05.mma (kind::f16, BF16 operands from shared
// memory, FP32 accumulators in tensor memory) computes [128 x 64] x [64 x 64]
// and [128 x 64] x [64 x 256]; the epilogues read the accumulators back with
// tcgen05.ld (thread i of the CTA owns row i, i.e. TMEM lane i), add the
// bias, apply GELU / take the top-1.  Layer 1 (K = 6) stays on the CUDA
// cores.  The hidden activations enter the tensor cores rounded to BF16.
//
// Operands use the no-swizzle K-major layout of 8 x 8 "core matrices" (8
// rows x 16 bytes, stored contiguously): element (row r, k) of a K = 64
// operand sits at byte ((r / 8) * 8 + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2,
// so core matrices adjacent along K are 128 bytes apart and 8-row groups
// 1024 bytes apart.  Every address a descriptor can reach stays inside the
// operand's own buffer whichever way those two strides are read.
namespace tc {

constexpr int M = 128;           // rays per tile (TMEM lanes)
constexpr int K = 64;            // hidden width = K of layers 2 and 3
constexpr int kTmemCols = 256;   // accumulator columns (N of layer 3)
constexpr unsigned kSpinLimit = 1u << 24;  // bounded mbarrier wait

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}
__device__ __forceinline__ uint32_t core_off(int r, int k) {
  return (uint32_t)(((r >> 3) * 8 + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}
// Shared-memory matrix descriptor: start, leading-dimension (K) byte
// offset, stride-dimension (8-row) byte offset, fixed field 0b001 at bit 46,
// no swizzle.
__device__ __forceinline__ uint64_t desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = (uint64_t)((saddr & 0x3FFFFu) >> 4);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}
// Instruction descriptor of kind::f16: D = F32, A = B = BF16, both K-major.
__host__ __device__ constexpr uint32_t idesc(int m, int n) {
  return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(n >> 3) << 17) |
         ((uint32_t)(m >> 4) << 24);
}
__device__ __forceinline__ void mma(uint32_t tmem, uint64_t a, uint64_t b, uint32_t id,
                                    uint32_t acc) {
  asm volatile(
      "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
      "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n" ::"r"(tmem),
      "l"(a), "l"(b), "r"(id), "r"(acc));
}
__device__ __forceinline__ void commit(void* mbar) {
  asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                   smem_u32(mbar))
               : "memory");
}
__device__ __forceinline__ bool wait_parity(void* mbar, uint32_t parity) {
  for (unsigned it = 0; it < kSpinLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n.reg .pred p;\nmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        "selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(done)
        : "r"(smem_u32(mbar)), "r"(parity)
        : "memory");
    if (done) return true;
  }
  return false;
}
// 16 consecutive FP32 accumulator columns of this thread's TMEM lane.
__device__ __forceinline__ void ld16(uint32_t taddr, float* v) {
  uint32_t r[16];
  asm volatile(
      "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,"
      "%14,%15}, [%16];\n"
      : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]),
        "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]),
        "=r"(r[14]), "=r"(r[15])
      : "r"(taddr));
  asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

struct __align__(1024) Smem {
  __nv_bfloat16 w3[256 * K];  // B of layer 3 (N = 256), core-matrix layout
  __nv_bfloat16 w2[64 * K];   // B of layer 2 (N = 64)
  __nv_bfloat16 a[M * K];     // A of layer 2, then of layer 3
  float w1[64 * IN], b1[64], b2[64], b3[256];
  unsigned long long mbar;
  uint32_t tmem_slot;
  int err;
};

}  // namespace tc

// Status bit of a tensor-core wait that ran out (the kernel then stops).
constexpr unsigned kMlpTimeout = 1u;

__global__ void __launch_bounds__(tc::M) infer_tc_kernel(const __nv_bfloat16* wb,
                                                          const float4* rays, long long n,
                                                          const float* box, int* cls,
                                                          float* logits, float min_prob,
                                                          unsigned* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw_tc[];
  tc::Smem& sm = *reinterpret_cast<tc::Smem*>(smem_raw_tc);
  const int tid = threadIdx.x, warp = tid >> 5;
  // stage the weights: W2, W3 into the core-matrix layout, the rest as floats
  for (int i = tid; i < 64 * tc::K; i += blockDim.x) {
    const int r = i / tc::K, k = i % tc::K;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(sm.w2) +
                                      tc::core_off(r, k)) = wb[OFF_W2 + i];
  }
  for (int i = tid; i < 256 * tc::K; i += blockDim.x) {
    const int r = i / tc::K, k = i % tc::K;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(sm.w3) +
                                      tc::core_off(r, k)) = wb[OFF_W3 + i];
  }
  for (int i = tid; i < 64 * IN; i += blockDim.x) sm.w1[i] = __bfloat162float(wb[OFF_W1 + i]);
  for (int i = tid; i < 64; i += blockDim.x) {
    sm.b1[i] = __bfloat162float(wb[OFF_B1 + i]);
    sm.b2[i] = __bfloat162float(wb[OFF_B2 + i]);
  }
  for (int i = tid; i < 256; i += blockDim.x) sm.b3[i] = __bfloat162float(wb[OFF_B3 + i]);
  if (tid == 0) {
    sm.err = 0;
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(tc::smem_u32(&sm.mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
  }
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     tc::smem_u32(&sm.tmem_slot)),
                 "r"(tc::kTmemCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = sm.tmem_slot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t a_addr = tc::smem_u32(sm.a), w2_addr = tc::smem_u32(sm.w2),
                 w3_addr = tc::smem_u32(sm.w3);
  float bx[6];
  for (int k = 0; k < 6; ++k) bx[k] = box[k];
  uint32_t phase = 0;
  for (long long t0 = (long long)blockIdx.x * tc::M; t0 < n; t0 += (long long)gridDim.x * tc::M) {
    const long long r = t0 + tid;
    // layer 1 on the CUDA cores: h1 = gelu(W1 x + b1) -> BF16 A tile
    float x[IN];
    if (r < n) {
      features(__ldg(&rays[2 * r]), __ldg(&rays[2 * r + 1]), bx, x);
    } else {
      for (int i = 0; i < IN; ++i) x[i] = 0.0f;
    }
    unsigned char* abytes = reinterpret_cast<unsigned char*>(sm.a);
#pragma unroll 8
    for (int o = 0; o < 64; ++o) {
      float acc = sm.b1[o];
#pragma unroll
      for (int i = 0; i < IN; ++i) acc += sm.w1[o * IN + i] * x[i];
      *reinterpret_cast<__nv_bfloat16*>(abytes + tc::core_off(tid, o)) =
          __float2bfloat16_rn(gelu(acc));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 2: [128 x 64] x [64 x 64] into TMEM columns 0..63
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < tc::K / 16; ++s)
        tc::mma(tmem, tc::desc(a_addr + s * 256, 128, 1024), tc::desc(w2_addr + s * 256, 128, 1024),
                tc::idesc(tc::M, 64), s > 0);
      tc::commit(&sm.mbar);
    }
    if (!tc::wait_parity(&sm.mbar, phase)) {
      if (tid == 0) atomicOr(status, kMlpTimeout);
      sm.err = 1;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (sm.err) break;
    // epilogue 2: h2 = gelu(acc + b2) -> BF16 A tile (layer 2 is done with it)
#pragma unroll
    for (int c = 0; c < 64; c += 16) {
      float v[16];
      tc::ld16(tmem + lane_base + c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j)
        *reinterpret_cast<__nv_bfloat16*>(abytes + tc::core_off(tid, c + j)) =
            __float2bfloat16_rn(gelu(v[j] + sm.b2[c + j]));
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    // layer 3: [128 x 64] x [64 x 256] into TMEM columns 0..255
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < tc::K / 16; ++s)
        tc::mma(tmem, tc::desc(a_addr + s * 256, 128, 1024), tc::desc(w3_addr + s * 256, 128, 1024),
                tc::idesc(tc::M, 256), s > 0);
      tc::commit(&sm.mbar);
    }
    if (!tc::wait_parity(&sm.mbar, phase)) {
      if (tid == 0) atomicOr(status, kMlpTimeout);
      sm.err = 1;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (sm.err) break;
    // epilogue 3: logits = acc + b3; top-1 with the optional abstention
    float best = -INFINITY, se = 0.0f;
    int bi = 0;
    for (int c = 0; c < 256; c += 16) {
      float v[16];
      tc::ld16(tmem + lane_base + c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float z = v[j] + sm.b3[c + j];
        if (logits && r < n) logits[r * OUT + c + j] = z;
        if (z > best) {
          if (min_prob > 0.0f) se = se * expf(best - z) + 1.0f;
          best = z;
          bi = c + j;
        } else if (min_prob > 0.0f) {
          se += expf(z - best);
        }
      }
    }
    if (r < n) cls[r] = (min_prob > 0.0f && se * min_prob > 1.0f) ? -1 : bi;
    // the next tile's layer 1 overwrites the A tile and layer 2 the
    // accumulators only after every thread has read them
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem),
                 "r"(tc::kTmemCols));
}

// ------------------------------------------------ tensor-core training --
// The training step's contractions on the tensor cores, with BF16 operands
// and FP32 accumulation, in the K-major no-swizzle layout of the inference
// kernel generalised to any K (a multiple of 16): element (r, k) of an
// operand with K columns sits at byte
// ((r / 8) * (K / 8) + k / 8) * 128 + (r % 8) * 16 + (k % 8) * 2, so core
// matrices adjacent along K are 128 bytes apart and 8-row groups K * 16
// bytes apart.  Three kernels: the forward pass that keeps A1, A2 and dZ
// (layers 2 and 3 as products, as in inference); the weight gradients
// dW += dA^T H over a batch slice (a column of ones in H gives the bias
// gradient in the same product); and the hidden backward
// dA_prev = (dA W) * gelu'(A_prev).
namespace tc {

__device__ __forceinline__ uint32_t core_off_k(int r, int k, int K) {
  return (uint32_t)(((r >> 3) * (K >> 3) + (k >> 3)) * 128 + (r & 7) * 16 + (k & 7) * 2);
}

__device__ __forceinline__ void put_bf16(unsigned char* base, uint32_t off, float v) {
  *reinterpret_cast<__nv_bfloat16*>(base + off) = __float2bfloat16_rn(v);
}

// Sequence point between threads' shared-memory writes and the tensor
// cores' reads (or their TMEM writes and the threads' reads).
__device__ __forceinline__ void sync_async() {
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

__device__ __forceinline__ void tmem_alloc(uint32_t* slot, uint32_t cols) {
  asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                   smem_u32(slot)),
               "r"(cols));
  asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
}

__device__ __forceinline__ void tmem_free(uint32_t tmem, uint32_t cols) {
  asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(cols));
}

__device__ __forceinline__ void mbar_init(void* mbar) {
  asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_u32(mbar)));
  asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}

}  // namespace tc

// Training forward on the tensor cores: A1 and A2 (pre-activations, FP32),
// dZ = (softmax(z) - onehot(y)) / B and the mean loss, for a batch.  The
// hidden activations enter the products rounded to BF16, as in inference.
__global__ void __launch_bounds__(tc::M) train_fwd_tc_kernel(
    const __nv_bfloat16* wb, const float4* rays, const int* labels, long long B, const float* box,
    float* A1, float* A2, float* dZ, float* loss, unsigned* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw_tc[];
  tc::Smem& sm = *reinterpret_cast<tc::Smem*>(smem_raw_tc);
  const int tid = threadIdx.x, warp = tid >> 5;
  for (int i = tid; i < 64 * tc::K; i += blockDim.x) {
    const int r = i / tc::K, k = i % tc::K;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(sm.w2) +
                                      tc::core_off(r, k)) = wb[OFF_W2 + i];
  }
  for (int i = tid; i < 256 * tc::K; i += blockDim.x) {
    const int r = i / tc::K, k = i % tc::K;
    *reinterpret_cast<__nv_bfloat16*>(reinterpret_cast<unsigned char*>(sm.w3) +
                                      tc::core_off(r, k)) = wb[OFF_W3 + i];
  }
  for (int i = tid; i < 64 * IN; i += blockDim.x) sm.w1[i] = __bfloat162float(wb[OFF_W1 + i]);
  for (int i = tid; i < 64; i += blockDim.x) {
    sm.b1[i] = __bfloat162float(wb[OFF_B1 + i]);
    sm.b2[i] = __bfloat162float(wb[OFF_B2 + i]);
  }
  for (int i = tid; i < 256; i += blockDim.x) sm.b3[i] = __bfloat162float(wb[OFF_B3 + i]);
  if (tid == 0) {
    sm.err = 0;
    tc::mbar_init(&sm.mbar);
  }
  if (warp == 0) tc::tmem_alloc(&sm.tmem_slot, tc::kTmemCols);
  tc::sync_async();
  const uint32_t tmem = sm.tmem_slot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t a_addr = tc::smem_u32(sm.a), w2_addr = tc::smem_u32(sm.w2),
                 w3_addr = tc::smem_u32(sm.w3);
  float bx[6];
  for (int k = 0; k < 6; ++k) bx[k] = box[k];
  const float invB = 1.0f / (float)B;
  float lsum = 0.0f;
  uint32_t phase = 0;
  unsigned char* abytes = reinterpret_cast<unsigned char*>(sm.a);
  for (long long t0 = (long long)blockIdx.x * tc::M; t0 < B; t0 += (long long)gridDim.x * tc::M) {
    const long long r = t0 + tid;
    const bool live = r < B;
    float x[IN];
    if (live) {
      features(__ldg(&rays[2 * r]), __ldg(&rays[2 * r + 1]), bx, x);
    } else {
      for (int i = 0; i < IN; ++i) x[i] = 0.0f;
    }
#pragma unroll 8
    for (int o = 0; o < 64; ++o) {
      float acc = sm.b1[o];
#pragma unroll
      for (int i = 0; i < IN; ++i) acc += sm.w1[o * IN + i] * x[i];
      if (live) A1[r * H + o] = acc;
      tc::put_bf16(abytes, tc::core_off(tid, o), gelu(acc));
    }
    tc::sync_async();
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < tc::K / 16; ++s)
        tc::mma(tmem, tc::desc(a_addr + s * 256, 128, 1024), tc::desc(w2_addr + s * 256, 128, 1024),
                tc::idesc(tc::M, 64), s > 0);
      tc::commit(&sm.mbar);
    }
    if (!tc::wait_parity(&sm.mbar, phase)) {
      if (tid == 0) atomicOr(status, kMlpTimeout);
      sm.err = 1;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (sm.err) break;
#pragma unroll
    for (int c = 0; c < 64; c += 16) {
      float v[16];
      tc::ld16(tmem + lane_base + c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float a2 = v[j] + sm.b2[c + j];
        if (live) A2[r * H + c + j] = a2;
        tc::put_bf16(abytes, tc::core_off(tid, c + j), gelu(a2));
      }
    }
    tc::sync_async();
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < tc::K / 16; ++s)
        tc::mma(tmem, tc::desc(a_addr + s * 256, 128, 1024), tc::desc(w3_addr + s * 256, 128, 1024),
                tc::idesc(tc::M, 256), s > 0);
      tc::commit(&sm.mbar);
    }
    if (!tc::wait_parity(&sm.mbar, phase)) {
      if (tid == 0) atomicOr(status, kMlpTimeout);
      sm.err = 1;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (sm.err) break;
    // softmax over the 256 logits of this thread's row: max, then the sum
    // of exponentials, then dZ; the label's logit is picked on the way
    const int y = live ? labels[r] : 0;
    float m = -INFINITY, zy = 0.0f;
    for (int c = 0; c < 256; c += 16) {
      float v[16];
      tc::ld16(tmem + lane_base + c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) {
        const float z = v[j] + sm.b3[c + j];
        m = fmaxf(m, z);
        if (c + j == y) zy = z;
      }
    }
    float se = 0.0f;
    for (int c = 0; c < 256; c += 16) {
      float v[16];
      tc::ld16(tmem + lane_base + c, v);
#pragma unroll
      for (int j = 0; j < 16; ++j) se += expf(v[j] + sm.b3[c + j] - m);
    }
    const float inv = 1.0f / se;
    for (int c = 0; c < 256; c += 16) {
      float v[16];
      tc::ld16(tmem + lane_base + c, v);
      if (live) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          dZ[r * OUT + c + j] =
              (expf(v[j] + sm.b3[c + j] - m) * inv - (c + j == y ? 1.0f : 0.0f)) * invB;
      }
    }
    if (live) lsum += (logf(se) + m) - zy;
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  __shared__ float red[tc::M];
  red[tid] = lsum;
  __syncthreads();
  for (int st = tc::M / 2; st > 0; st >>= 1) {
    if (tid < st) red[tid] += red[tid + st];
    __syncthreads();
  }
  if (tid == 0) atomicAdd(loss, red[0] * invB);
  if (warp == 0) tc::tmem_free(tmem, tc::kTmemCols);
}

// Weight gradients over a batch slice: dW[o][i] += sum_b dA[b][o] Hin[b][i]
// and db[o] += sum_b dA[b][o], as one product per 64-ray chunk: A = dA^T
// (128 outputs of this CTA's tile x 64 rays), B = [Hin | 1 | 0]^T (NP x 64,
// NP = I + 1 rounded up to 16), both BF16; Hin = gelu(Asrc) (act 1), Asrc
// (act 0) or the ray features (act 2, Asrc = rays).  The FP32 accumulator
// stays in TMEM over the slice and is added to dW / db at the end.
constexpr int kGradChunk = 64;

template <int NP>
struct GradSmem {
  __nv_bfloat16 a[tc::M * kGradChunk];
  __nv_bfloat16 b[NP * kGradChunk];
  unsigned long long mbar;
  uint32_t tmem_slot;
  int err;
};

template <int NP>
__global__ void __launch_bounds__(tc::M) grad_tc_kernel(const float* dA, int O, const float* Asrc,
                                                        int I, int act, const float* box,
                                                        long long B, long long slice, float* dW,
                                                        float* db, unsigned* status) {
  constexpr uint32_t kCols = NP <= 32 ? 32 : (NP <= 64 ? 64 : (NP <= 128 ? 128 : 256));
  __shared__ __align__(1024) GradSmem<NP> sm;
  const int tid = threadIdx.x, warp = tid >> 5;
  const int o0 = blockIdx.y * tc::M;
  const long long b_begin = (long long)blockIdx.x * slice;
  const long long b_end = b_begin + slice < B ? b_begin + slice : B;
  if (tid == 0) {
    sm.err = 0;
    tc::mbar_init(&sm.mbar);
  }
  if (warp == 0) tc::tmem_alloc(&sm.tmem_slot, kCols);
  tc::sync_async();
  const uint32_t tmem = sm.tmem_slot;
  float bx[6] = {0, 0, 0, 1, 1, 1};
  if (act == 2)
    for (int k = 0; k < 6; ++k) bx[k] = box[k];
  unsigned char* ab = reinterpret_cast<unsigned char*>(sm.a);
  unsigned char* bb = reinterpret_cast<unsigned char*>(sm.b);
  const uint32_t a_addr = tc::smem_u32(sm.a), b_addr = tc::smem_u32(sm.b);
  uint32_t phase = 0;
  bool first = true;
  for (long long c0 = b_begin; c0 < b_end; c0 += kGradChunk) {
    // A: element (o, k) = dA[c0 + k][o0 + o]; consecutive threads take
    // consecutive outputs of one ray (coalesced reads)
    for (int e = tid; e < tc::M * kGradChunk; e += tc::M) {
      const int o = e % tc::M, k = e / tc::M;
      const long long b = c0 + k;
      const float v = (b < b_end && o0 + o < O) ? dA[b * O + o0 + o] : 0.0f;
      tc::put_bf16(ab, tc::core_off_k(o, k, kGradChunk), v);
    }
    // B: element (i, k) = Hin[c0 + k][i] for i < I, 1 at i = I (a ray in
    // the slice), 0 beyond
    for (int e = tid; e < NP * kGradChunk; e += tc::M) {
      const int i = e % NP, k = e / NP;
      const long long b = c0 + k;
      float v = 0.0f;
      if (b < b_end) {
        if (i < I) {
          if (act == 2) {
            const float4* rr = reinterpret_cast<const float4*>(Asrc) + 2 * b;
            float x[IN];
            features(rr[0], rr[1], bx, x);
            v = x[i];
          } else {
            const float a = Asrc[b * I + i];
            v = act ? gelu(a) : a;
          }
        } else if (i == I) {
          v = 1.0f;
        }
      }
      tc::put_bf16(bb, tc::core_off_k(i, k, kGradChunk), v);
    }
    tc::sync_async();
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < kGradChunk / 16; ++s)
        tc::mma(tmem, tc::desc(a_addr + s * 256, 128, (kGradChunk / 8) * 128),
                tc::desc(b_addr + s * 256, 128, (kGradChunk / 8) * 128), tc::idesc(tc::M, NP),
                (first && s == 0) ? 0u : 1u);
      tc::commit(&sm.mbar);
    }
    first = false;
    if (!tc::wait_parity(&sm.mbar, phase)) {
      if (tid == 0) atomicOr(status, kMlpTimeout);
      sm.err = 1;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (sm.err) break;
  }
  if (!sm.err && !first) {
    // thread t holds output o0 + t (TMEM lane t)
    const int o = o0 + tid;
    const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
#pragma unroll
    for (int c = 0; c < NP; c += 16) {
      float v[16];
      tc::ld16(tmem + lane_base + c, v);
      if (o < O) {
#pragma unroll
        for (int j = 0; j < 16; ++j) {
          const int i = c + j;
          if (i < I) atomicAdd(&dW[o * I + i], v[j]);
          else if (i == I) atomicAdd(&db[o], v[j]);
        }
      }
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0) tc::tmem_free(tmem, kCols);
}

// Hidden backward on the tensor cores: dAprev[b][i] = (sum_o dA[b][o]
// W[o][i]) * gelu'(Aprev[b][i]) per tile of 128 rays: A = dA (128 x O, BF16),
// B = W^T (64 x O, from the BF16 weights), FP32 accumulation.
template <int O>
struct BackSmem {
  __nv_bfloat16 a[tc::M * O];
  __nv_bfloat16 w[64 * O];
  unsigned long long mbar;
  uint32_t tmem_slot;
  int err;
};

template <int O>
__global__ void __launch_bounds__(tc::M) back_tc_kernel(const float* dA,
                                                        const __nv_bfloat16* wb, int off_w,
                                                        const float* Aprev, long long B,
                                                        float* dAprev, unsigned* status) {
  extern __shared__ __align__(1024) unsigned char smem_raw_tc[];
  BackSmem<O>& sm = *reinterpret_cast<BackSmem<O>*>(smem_raw_tc);
  const int tid = threadIdx.x, warp = tid >> 5;
  unsigned char* ab = reinterpret_cast<unsigned char*>(sm.a);
  unsigned char* wbytes = reinterpret_cast<unsigned char*>(sm.w);
  // W^T: element (i, o) = W[o][i]
  for (int e = tid; e < 64 * O; e += tc::M) {
    const int o = e / 64, i = e % 64;
    *reinterpret_cast<__nv_bfloat16*>(wbytes + tc::core_off_k(i, o, O)) = wb[off_w + o * 64 + i];
  }
  if (tid == 0) {
    sm.err = 0;
    tc::mbar_init(&sm.mbar);
  }
  if (warp == 0) tc::tmem_alloc(&sm.tmem_slot, 64);
  tc::sync_async();
  const uint32_t tmem = sm.tmem_slot;
  const uint32_t lane_base = (uint32_t)(warp * 32) << 16;
  const uint32_t a_addr = tc::smem_u32(sm.a), w_addr = tc::smem_u32(sm.w);
  uint32_t phase = 0;
  for (long long t0 = (long long)blockIdx.x * tc::M; t0 < B; t0 += (long long)gridDim.x * tc::M) {
    // A: element (b, o) = dA[t0 + b][o]; consecutive threads, consecutive o
    for (int e = tid; e < tc::M * O; e += tc::M) {
      const int b = e / O, o = e % O;
      const long long r = t0 + b;
      tc::put_bf16(ab, tc::core_off_k(b, o, O), r < B ? dA[r * O + o] : 0.0f);
    }
    tc::sync_async();
    if (tid == 0) {
#pragma unroll
      for (int s = 0; s < O / 16; ++s)
        tc::mma(tmem, tc::desc(a_addr + s * 256, 128, (O / 8) * 128),
                tc::desc(w_addr + s * 256, 128, (O / 8) * 128), tc::idesc(tc::M, 64), s > 0);
      tc::commit(&sm.mbar);
    }
    if (!tc::wait_parity(&sm.mbar, phase)) {
      if (tid == 0) atomicOr(status, kMlpTimeout);
      sm.err = 1;
    }
    phase ^= 1u;
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    __syncthreads();
    if (sm.err) break;
    const long long r = t0 + tid;
#pragma unroll
    for (int c = 0; c < 64; c += 16) {
      float v[16];
      tc::ld16(tmem + lane_base + c, v);
      if (r < B) {
#pragma unroll
        for (int j = 0; j < 16; ++j)
          dAprev[r * H + c + j] = v[j] * gelu_grad(Aprev[r * H + c + j]);
      }
    }
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  }
  if (warp == 0) tc::tmem_free(tmem, 64);
}

int num_sms() {
  static std::once_flag f;
  static int sms = 0;
  std::call_once(f, [] {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  });
  return sms > 0 ? sms : 1;
}

}  // namespace mlpk

#define CUDA_OK(call)                                                        \
  do {                                                                       \
    cudaError_t e_ = (call);                                                 \
    if (e_ != cudaSuccess)                                                   \
      fail(SC_ERR_CUDA, "%s failed: %s", #call, cudaGetErrorString(e_));    \
  } while (0)

#define SC_TRY \
  try {        \
    clear_error();
#define SC_CATCH                            \
  }                                         \
  catch (const Error& e) {                  \
    set_error("%s", e.msg.c_str());         \
    return e.code;                          \
  }                                         \
  catch (...) {                             \
    set_error("unexpected internal error"); \
    return SC_ERR_STATE;                    \
  }

namespace {

constexpr size_t kSmemW = sizeof(mlpk::SmemW);

void set_smem(const void* k) {
  CUDA_OK(cudaFuncSetAttribute(k, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmemW));
}

int grid_for(long long n, int threads) {
  long long g = (n + threads - 1) / threads;
  const long long cap = (long long)mlpk::num_sms() * 2;
  if (g > cap) g = cap;
  return (int)(g > 0 ? g : 1);
}

void check_box(const float* box) {
  if (!box) fail(SC_ERR_ARG, "mlp: NULL scene box");
}

}  // namespace

extern "C" {

int sc_mlp_num_params(void) { return mlpk::P; }

size_t sc_mlp_train_workspace_bytes(int64_t batch) {
  return (size_t)batch * (3 * mlpk::H + mlpk::OUT) * 4 + 256;
}

sc_status sc_mlp_to_bf16(const float* d_w, void* d_wb, void* stream) {
  SC_TRY
  if (!d_w || !d_wb) fail(SC_ERR_ARG, "sc_mlp_to_bf16: NULL argument");
  mlpk::to_bf16_kernel<<<(mlpk::P + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      d_w, reinterpret_cast<__nv_bfloat16*>(d_wb));
  CUDA_OK(cudaGetLastError());
  return SC_OK;
  SC_CATCH
}

sc_status sc_mlp_forward(const void* d_wb, const float* d_rays, int64_t n, const float* d_box,
                         int32_t* d_cls, float* d_logits, float min_prob, void* stream) {
  SC_TRY
  check_box(d_box);
  if (n < 0 || (n > 0 && (!d_wb || !d_rays || !d_cls))) fail(SC_ERR_ARG, "sc_mlp_forward: bad args");
  if (n == 0) return SC_OK;
  set_smem((const void*)mlpk::infer_kernel);
  mlpk::infer_kernel<<<grid_for(n, mlpk::kThreads), mlpk::kThreads, kSmemW,
                       reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const __nv_bfloat16*>(d_wb), reinterpret_cast<const float4*>(d_rays), n,
      d_box, d_cls, d_logits, min_prob);
  CUDA_OK(cudaGetLastError());
  return SC_OK;
  SC_CATCH
}

sc_status sc_mlp_forward_tc(const void* d_wb, const float* d_rays, int64_t n,
                            const float* d_box, int32_t* d_cls, float* d_logits, float min_prob,
                            void* d_status, void* stream) {
  SC_TRY
  check_box(d_box);
  if (n < 0 || (n > 0 && (!d_wb || !d_rays || !d_cls || !d_status)))
    fail(SC_ERR_ARG, "sc_mlp_forward_tc: bad args");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  CUDA_OK(cudaMemsetAsync(d_status, 0, sizeof(unsigned), st));
  if (n == 0) return SC_OK;
  const size_t smem = sizeof(mlpk::tc::Smem);
  CUDA_OK(cudaFuncSetAttribute((const void*)mlpk::infer_tc_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
  long long tiles = (n + mlpk::tc::M - 1) / mlpk::tc::M;
  // two CTAs per SM share its 512 TMEM columns
  const long long cap = 2LL * mlpk::num_sms();
  const unsigned grid = (unsigned)(tiles < cap ? tiles : cap);
  mlpk::infer_tc_kernel<<<grid, mlpk::tc::M, smem, st>>>(
      reinterpret_cast<const __nv_bfloat16*>(d_wb), reinterpret_cast<const float4*>(d_rays), n,
      d_box, d_cls, d_logits, min_prob, reinterpret_cast<unsigned*>(d_status));
  CUDA_OK(cudaGetLastError());
  return SC_OK;
  SC_CATCH
}

sc_status sc_mlp_grad(const void* d_wb, const float* d_rays, const int32_t* d_labels,
                      int64_t batch, const float* d_box, float* d_grad, float* d_loss,
                      void* d_ws, size_t ws_bytes, void* stream) {
  SC_TRY
  check_box(d_box);
  if (batch <= 0 || !d_wb || !d_rays || !d_labels || !d_grad || !d_loss || !d_ws)
    fail(SC_ERR_ARG, "sc_mlp_grad: bad arguments");
  if (ws_bytes < sc_mlp_train_workspace_bytes(batch)) fail(SC_ERR_ARG, "sc_mlp_grad: workspace too small");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  using namespace mlpk;
  float* A1 = reinterpret_cast<float*>(d_ws);
  float* A2 = A1 + batch * H;
  float* dZ = A2 + batch * H;
  const __nv_bfloat16* wb = reinterpret_cast<const __nv_bfloat16*>(d_wb);
  CUDA_OK(cudaMemsetAsync(d_loss, 0, sizeof(float), st));
  set_smem((const void*)train_fwd_kernel);
  train_fwd_kernel<<<grid_for(batch, kThreads), kThreads, kSmemW, st>>>(
      wb, reinterpret_cast<const float4*>(d_rays), d_labels, batch, d_box, A1, A2, dZ, d_loss);
  CUDA_OK(cudaGetLastError());
  // layer 3: dW3 = dZ^T h2, db3
  const long long slice = 512;  // batch rows per split-K block
  const unsigned nsl = (unsigned)((batch + slice - 1) / slice);
  grad_w_kernel<<<dim3(nsl, OUT / TG, H / TG), 256, 0, st>>>(dZ, OUT, A2, H, 1, d_box, batch,
                                                              slice, d_grad + OFF_W3,
                                                              d_grad + OFF_B3);
  CUDA_OK(cudaGetLastError());
  // dA2 = (dZ W3) * gelu'(A2), after dZ in the workspace
  float* dAh = dZ + batch * OUT;
  CUDA_OK(cudaFuncSetAttribute((const void*)back_hidden_kernel<OUT>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, OUT * H * 4));
  back_hidden_kernel<OUT><<<grid_for(batch, kThreads), kThreads, OUT * H * 4, st>>>(
      dZ, wb, OFF_W3, A2, batch, dAh);
  CUDA_OK(cudaGetLastError());
  // layer 2: dW2 = dA2^T h1, db2
  grad_w_kernel<<<dim3(nsl, H / TG, H / TG), 256, 0, st>>>(dAh, H, A1, H, 1, d_box, batch, slice,
                                                            d_grad + OFF_W2, d_grad + OFF_B2);
  CUDA_OK(cudaGetLastError());
  // dA1 = (dA2 W2) * gelu'(A1) -> into A2 (no longer needed)
  back_hidden_kernel<H><<<grid_for(batch, kThreads), kThreads, H * H * 4, st>>>(
      dAh, wb, OFF_W2, A1, batch, A2);
  CUDA_OK(cudaGetLastError());
  // layer 1: dW1 = dA1^T x, db1
  grad_w_kernel<<<dim3(nsl, H / TG, 1), 256, 0, st>>>(A2, H, d_rays, IN, 2, d_box, batch, slice,
                                                       d_grad + OFF_W1, d_grad + OFF_B1);
  CUDA_OK(cudaGetLastError());
  return SC_OK;
  SC_CATCH
}

sc_status sc_mlp_grad_tc(const void* d_wb, const float* d_rays, const int32_t* d_labels,
                         int64_t batch, const float* d_box, float* d_grad, float* d_loss,
                         void* d_ws, size_t ws_bytes, void* d_status, void* stream) {
  SC_TRY
  check_box(d_box);
  if (batch <= 0 || !d_wb || !d_rays || !d_labels || !d_grad || !d_loss || !d_ws || !d_status)
    fail(SC_ERR_ARG, "sc_mlp_grad_tc: bad arguments");
  if (ws_bytes < sc_mlp_train_workspace_bytes(batch))
    fail(SC_ERR_ARG, "sc_mlp_grad_tc: workspace too small");
  cudaStream_t st = reinterpret_cast<cudaStream_t>(stream);
  using namespace mlpk;
  float* A1 = reinterpret_cast<float*>(d_ws);
  float* A2 = A1 + batch * H;
  float* dZ = A2 + batch * H;
  float* dAh = dZ + batch * OUT;
  unsigned* status = reinterpret_cast<unsigned*>(d_status);
  const __nv_bfloat16* wb = reinterpret_cast<const __nv_bfloat16*>(d_wb);
  CUDA_OK(cudaMemsetAsync(d_loss, 0, sizeof(float), st));
  // forward: A1, A2, dZ and the loss (two CTAs per SM share its TMEM)
  const size_t fsm = sizeof(tc::Smem);
  CUDA_OK(cudaFuncSetAttribute((const void*)train_fwd_tc_kernel,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)fsm));
  const long long tiles = (batch + tc::M - 1) / tc::M, cap = 2LL * num_sms();
  train_fwd_tc_kernel<<<(unsigned)(tiles < cap ? tiles : cap), tc::M, fsm, st>>>(
      wb, reinterpret_cast<const float4*>(d_rays), d_labels, batch, d_box, A1, A2, dZ, d_loss,
      status);
  CUDA_OK(cudaGetLastError());
  const long long slice = 256;  // rays per split-K CTA of the weight gradients
  const unsigned nsl = (unsigned)((batch + slice - 1) / slice);
  // layer 3: dW3 = dZ^T gelu(A2), db3
  grad_tc_kernel<80><<<dim3(nsl, OUT / tc::M), tc::M, 0, st>>>(
      dZ, OUT, A2, H, 1, d_box, batch, slice, d_grad + OFF_W3, d_grad + OFF_B3, status);
  CUDA_OK(cudaGetLastError());
  // dA2 = (dZ W3) * gelu'(A2)
  const size_t bs3 = sizeof(BackSmem<OUT>), bs2 = sizeof(BackSmem<H>);
  CUDA_OK(cudaFuncSetAttribute((const void*)back_tc_kernel<OUT>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs3));
  CUDA_OK(cudaFuncSetAttribute((const void*)back_tc_kernel<H>,
                               cudaFuncAttributeMaxDynamicSharedMemorySize, (int)bs2));
  back_tc_kernel<OUT><<<(unsigned)(tiles < cap ? tiles : cap), tc::M, bs3, st>>>(
      dZ, wb, OFF_W3, A2, batch, dAh, status);
  CUDA_OK(cudaGetLastError());
  // layer 2: dW2 = dA2^T gelu(A1), db2
  grad_tc_kernel<80><<<dim3(nsl, 1), tc::M, 0, st>>>(dAh, H, A1, H, 1, d_box, batch, slice,
                                                     d_grad + OFF_W2, d_grad + OFF_B2, status);
  CUDA_OK(cudaGetLastError());
  // dA1 = (dA2 W2) * gelu'(A1), into A2 (no longer needed)
  back_tc_kernel<H><<<(unsigned)(tiles < cap ? tiles : cap), tc::M, bs2, st>>>(
      dAh, wb, OFF_W2, A1, batch, A2, status);
  CUDA_OK(cudaGetLastError());
  // layer 1: dW1 = dA1^T x, db1
  grad_tc_kernel<16><<<dim3(nsl, 1), tc::M, 0, st>>>(A2, H, d_rays, IN, 2, d_box, batch, slice,
                                                     d_grad + OFF_W1, d_grad + OFF_B1, status);
  CUDA_OK(cudaGetLastError());
  return SC_OK;
  SC_CATCH
}

sc_status sc_mlp_adam(float* d_w, void* d_wb, float* d_grad, float* d_m, float* d_v, int step,
                      float lr, float beta1, float beta2, float eps, void* stream) {
  SC_TRY
  if (!d_w || !d_wb || !d_grad || !d_m || !d_v || step < 1) fail(SC_ERR_ARG, "sc_mlp_adam: bad args");
  const float bc1 = 1.0f / (1.0f - std::pow(beta1, (float)step));
  const float bc2 = 1.0f / (1.0f - std::pow(beta2, (float)step));
  mlpk::adam_kernel<<<(mlpk::P + 255) / 256, 256, 0, reinterpret_cast<cudaStream_t>(stream)>>>(
      d_w, reinterpret_cast<__nv_bfloat16*>(d_wb), d_grad, d_m, d_v, lr, beta1, beta2, eps, bc1,
      bc2);
  CUDA_OK(cudaGetLastError());
  return SC_OK;
  SC_CATCH
}

sc_status sc_mlp_gather(const float* d_rays, const int32_t* d_labels, int64_t n, uint64_t key,
                        int64_t start, int64_t batch, float* d_out_rays, int32_t* d_out_labels,
                        void* stream) {
  SC_TRY
  if (n < 1 || n > (int64_t)0x7FFFFFFF || start < 0 || batch < 0 || start + batch > n)
    fail(SC_ERR_ARG, "sc_mlp_gather: need 0 <= start, start + batch <= n < 2^31");
  if (batch > 0 && (!d_rays || !d_labels || !d_out_rays || !d_out_labels))
    fail(SC_ERR_ARG, "sc_mlp_gather: NULL buffer");
  if ((reinterpret_cast<uintptr_t>(d_rays) & 15) || (reinterpret_cast<uintptr_t>(d_out_rays) & 15))
    fail(SC_ERR_ARG, "sc_mlp_gather: rays must be 16-byte aligned");
  if (batch == 0) return SC_OK;
  int bits = 1;
  while (bits < 31 && (int64_t(1) << bits) < n) ++bits;
  const int h = (bits + 1) / 2;
  // four round keys from the 64-bit key (SplitMix64 steps)
  uint64_t z = key;
  uint32_t k[4];
  for (int r = 0; r < 4; ++r) {
    z += 0x9E3779B97F4A7C15ull;
    uint64_t x = z;
    x = (x ^ (x >> 30)) * 0xBF58476D1CE4E5B9ull;
    x = (x ^ (x >> 27)) * 0x94D049BB133111EBull;
    k[r] = (uint32_t)(x ^ (x >> 31));
  }
  mlpk::gather_kernel<<<(unsigned)((batch + 255) / 256), 256, 0,
                        reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const float4*>(d_rays), d_labels, n, h, make_uint4(k[0], k[1], k[2], k[3]),
      start, batch, reinterpret_cast<float4*>(d_out_rays), d_out_labels);
  CUDA_OK(cudaGetLastError());
  return SC_OK;
  SC_CATCH
}

sc_status sc_mlp_labels(const float* d_rays, const void* d_hits, int64_t n,
                        const uint8_t* d_class_of_tri, float* d_out_rays, int32_t* d_out_labels,
                        uint32_t* d_count, int64_t cap, void* stream) {
  SC_TRY
  if (n < 0 || (n > 0 && (!d_rays || !d_hits || !d_class_of_tri || !d_out_rays || !d_out_labels ||
                          !d_count)))
    fail(SC_ERR_ARG, "sc_mlp_labels: bad arguments");
  if (n == 0) return SC_OK;
  mlpk::labels_kernel<<<(unsigned)((n + 255) / 256), 256, 0,
                        reinterpret_cast<cudaStream_t>(stream)>>>(
      reinterpret_cast<const float4*>(d_rays), reinterpret_cast<const float4*>(d_hits), n,
      d_class_of_tri, reinterpret_cast<float4*>(d_out_rays), d_out_labels, d_count, cap);
  CUDA_OK(cudaGetLastError());
  return SC_OK;
  SC_CATCH
}

}  // extern "C"
