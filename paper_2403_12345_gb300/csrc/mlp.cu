// Importance network for weight windows: a 4 -> 64 -> 64 -> 1 MLP (ReLU)
// with BF16 weights and FP32 accumulation, evaluated and trained by these
// kernels.  The 4-input and 1-output layers are too narrow for the tensor
// cores and run on the FP32 pipe; the 64 x 64 layer runs on the tensor cores:
//
// - inference (k_mlp_forward_tc): fifth-generation tensor cores.  A CTA of
//   four warps takes 128 samples at a time: layer 1 writes relu(z1) as BF16
//   into shared memory in the canonical K-major layout, one thread issues
//   four tcgen05.mma (M 128, N 64, K 16 each) into a TMEM accumulator and
//   commits them to an mbarrier, and each warp reads its 32 TMEM lanes
//   (rows) back for bias, ReLU and layer 3;
// - training (k_mlp_grad): mma.sync m16n8k16, each warp carrying 16 samples
//   through forward and backward in registers (the accumulator fragments of
//   one layer are the A fragments of the next).
//
// Parameter layout (also the C ABI's): W1[64][4], b1[64], W2[64][64]
// (row = output unit), b2[64], W3[64], b3.
#include <cuda_bf16.h>

#include <algorithm>

#include "device.cuh"
#include "mlp.h"

namespace gbmc {

namespace {

constexpr int H = kMlpHidden;
constexpr unsigned kAll = 0xffffffffu;
constexpr int kWarps = 8;   // warps per block: 128 samples per block step

// Weights as the kernels use them: the BF16 values, as fp32 for the narrow
// layers and as packed bf16 pairs (both orientations) for the 64 x 64 layer.
struct SmemNet {
    float W1[H * 4], b1[H], b2[H], W3[H], b3;
    __nv_bfloat16 W2[H * H];    // [out][in]
    __nv_bfloat16 W2T[H * H];   // [in][out]
};

__device__ __forceinline__ uint32_t pack2(float lo, float hi) {
    __nv_bfloat162 v = __floats2bfloat162_rn(lo, hi);
    return *reinterpret_cast<uint32_t*>(&v);
}

__device__ __forceinline__ void mma16816(float* d, const uint32_t* a, uint32_t b0, uint32_t b1) {
    asm volatile(
        "mma.sync.aligned.m16n8k16.row.col.f32.bf16.bf16.f32 "
        "{%0,%1,%2,%3}, {%4,%5,%6,%7}, {%8,%9}, {%0,%1,%2,%3};\n"
        : "+f"(d[0]), "+f"(d[1]), "+f"(d[2]), "+f"(d[3])
        : "r"(a[0]), "r"(a[1]), "r"(a[2]), "r"(a[3]), "r"(b0), "r"(b1));
}

// Load the BF16 weights into shared memory (block-wide).
__device__ void load_net(SmemNet& S, const __nv_bfloat16* __restrict__ w) {
    const __nv_bfloat16* W1 = w;
    const __nv_bfloat16* b1 = W1 + H * 4;
    const __nv_bfloat16* W2 = b1 + H;
    const __nv_bfloat16* b2 = W2 + H * H;
    const __nv_bfloat16* W3 = b2 + H;
    const __nv_bfloat16* b3 = W3 + H;
    for (int k = threadIdx.x; k < H * H; k += blockDim.x) {
        __nv_bfloat16 v = W2[k];
        S.W2[k] = v;
        S.W2T[(k % H) * H + k / H] = v;
    }
    for (int k = threadIdx.x; k < H * 4; k += blockDim.x) S.W1[k] = __bfloat162float(W1[k]);
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
        S.b1[k] = __bfloat162float(b1[k]);
        S.b2[k] = __bfloat162float(b2[k]);
        S.W3[k] = __bfloat162float(W3[k]);
    }
    if (threadIdx.x == 0) S.b3 = __bfloat162float(b3[0]);
    __syncthreads();
}

// Shared memory of the gradient kernel: the net, the block's gradient
// accumulators and, per warp, dz2^T and relu(z1)^T staged as bf16 for the
// tensor-core dW2 product.
struct GradSmem {
    SmemNet net;
    float gW1[H * 4], gb1[H], gW2[H * H], gb2[H], gW3[H], gb3, lsum;
    __nv_bfloat16 stage[kWarps][2][H * 16];
};

// Per-warp state of 16 samples (rows g and g+8 of each tile for this lane,
// g = lane / 4, t = lane % 4).  Tile j covers units 8j .. 8j+7; this lane
// holds units 8j + 2t and 8j + 2t + 1 of both rows.
struct Tile16 {
    float x[2][4];        // features of rows g, g+8
    float z1[8][4];       // layer-1 pre-activations, tile order (c0, c1: row g; c2, c3: row g+8)
    float z2[8][4];       // layer-2 pre-activations
    float out[2];         // network output of rows g, g+8
};

// Forward pass of the 16 samples whose features this lane loaded.
__device__ __forceinline__ void forward16(const SmemNet& S, Tile16& T) {
    int lane = threadIdx.x & 31;
    int t = lane & 3;
    // layer 1 (FP32): units 8j + 2t + {0, 1} for both rows
#pragma unroll
    for (int j = 0; j < 8; ++j)
#pragma unroll
        for (int e = 0; e < 4; ++e) {
            int u = 8 * j + 2 * t + (e & 1);
            int r = e >> 1;
            float s = S.b1[u];
#pragma unroll
            for (int i = 0; i < 4; ++i) s += S.W1[u * 4 + i] * T.x[r][i];
            T.z1[j][e] = s;
        }
    // layer 2 (tensor cores): A = relu(z1) as bf16, B = W2^T
    uint32_t a[4][4];
#pragma unroll
    for (int kk = 0; kk < 4; ++kk) {
        const float* lo = T.z1[2 * kk];
        const float* hi = T.z1[2 * kk + 1];
        a[kk][0] = pack2(fmaxf(lo[0], 0.f), fmaxf(lo[1], 0.f));
        a[kk][1] = pack2(fmaxf(lo[2], 0.f), fmaxf(lo[3], 0.f));
        a[kk][2] = pack2(fmaxf(hi[0], 0.f), fmaxf(hi[1], 0.f));
        a[kk][3] = pack2(fmaxf(hi[2], 0.f), fmaxf(hi[3], 0.f));
    }
    int g = lane >> 2;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        float d[4] = {0.f, 0.f, 0.f, 0.f};
        const uint32_t* w = reinterpret_cast<const uint32_t*>(S.W2 + (8 * j + g) * H);
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) mma16816(d, a[kk], w[8 * kk + t], w[8 * kk + 4 + t]);
        int u0 = 8 * j + 2 * t;
        T.z2[j][0] = d[0] + S.b2[u0];
        T.z2[j][1] = d[1] + S.b2[u0 + 1];
        T.z2[j][2] = d[2] + S.b2[u0];
        T.z2[j][3] = d[3] + S.b2[u0 + 1];
    }
    // layer 3 (FP32): partial dot products over this lane's units, summed
    // over the 4 lanes of the group
    float p0 = 0.f, p1 = 0.f;
#pragma unroll
    for (int j = 0; j < 8; ++j) {
        int u0 = 8 * j + 2 * t;
        p0 += S.W3[u0] * fmaxf(T.z2[j][0], 0.f) + S.W3[u0 + 1] * fmaxf(T.z2[j][1], 0.f);
        p1 += S.W3[u0] * fmaxf(T.z2[j][2], 0.f) + S.W3[u0 + 1] * fmaxf(T.z2[j][3], 0.f);
    }
    p0 += __shfl_xor_sync(kAll, p0, 1);
    p0 += __shfl_xor_sync(kAll, p0, 2);
    p1 += __shfl_xor_sync(kAll, p1, 1);
    p1 += __shfl_xor_sync(kAll, p1, 2);
    T.out[0] = p0 + S.b3;
    T.out[1] = p1 + S.b3;
}

__device__ __forceinline__ void load_features(const float* __restrict__ feat, int64_t n,
                                              int64_t base, Tile16& T) {
    int g = (threadIdx.x & 31) >> 2;
#pragma unroll
    for (int r = 0; r < 2; ++r) {
        int64_t s = base + g + 8 * r;
#pragma unroll
        for (int i = 0; i < 4; ++i) T.x[r][i] = s < n ? feat[s * 4 + i] : 0.f;
    }
}

// ---------------------------------------------------------------- tcgen05 forward
// Shared-memory matrix descriptor (tcgen05): start address, leading byte
// offset (between core matrices along K), stride byte offset (between
// 8-row groups along M or N), all in 16-byte units; descriptor version 1;
// no swizzle.  A core matrix is 8 rows x 16 bytes, rows 16 bytes apart.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr & 0x3FFFFu) >> 4) | ((uint64_t)(lbo >> 4) << 16) |
           ((uint64_t)(sbo >> 4) << 32) | (1ull << 46);
}

// Instruction descriptor, kind::f16: D f32, A and B bf16, both K-major,
// N >> 3 at bit 17, M >> 4 at bit 24.
constexpr uint32_t kTcM = 128, kTcN = 64;
constexpr uint32_t kTcIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((kTcN >> 3) << 17) |
                              ((kTcM >> 4) << 24);
constexpr uint32_t kTcCols = 64;           // TMEM columns: the 128 x 64 f32 accumulator
constexpr uint32_t kTileBytes = 128 * 64 * 2;   // A: 128 rows x 64 bf16
constexpr uint32_t kWBytes = 64 * 64 * 2;       // B: W2, 64 rows (out) x 64 bf16 (in)
constexpr uint32_t kTcSpin = 1u << 22;     // mbarrier polls before giving up

struct TcNet {
    float W1[H * 4], b1[H], b2[H], W3[H], b3;
};
constexpr size_t kBarOff = (kTileBytes + kWBytes + sizeof(TcNet) + 7) & ~(size_t)7;

// Byte offset of element (row, k) of a 64-wide K-major bf16 operand in the
// canonical no-swizzle layout with K core matrices 128 bytes apart and row
// groups 1024 bytes apart.
__device__ __forceinline__ uint32_t kmajor_off(uint32_t row, uint32_t k) {
    return (row >> 3) * 1024u + (k >> 3) * 128u + (row & 7u) * 16u + (k & 7u) * 2u;
}

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

// Polls the mbarrier for the completion of `phase`, at most kTcSpin times.
__device__ __forceinline__ bool wait_phase(uint64_t* mbar, uint32_t phase) {
    uint32_t done = 0;
    for (uint32_t spin = 0; spin < kTcSpin && !done; ++spin)
        asm volatile(
            "{\n.reg .pred P;\nmbarrier.try_wait.parity.shared::cta.b64 P, [%1], %2;\n"
            "selp.u32 %0, 1, 0, P;\n}\n"
            : "=r"(done) : "r"(smem_u32(mbar)), "r"(phase) : "memory");
    return done != 0;
}

__global__ void __launch_bounds__(128) k_mlp_forward_tc(const __nv_bfloat16* __restrict__ w,
                                                        const float* __restrict__ feat, int64_t n,
                                                        float* __restrict__ out,
                                                        int* __restrict__ err) {
    extern __shared__ __align__(1024) unsigned char sm[];
    unsigned char* A = sm;                       // 16 KB
    unsigned char* B = sm + kTileBytes;          // 8 KB
    TcNet& S = *reinterpret_cast<TcNet*>(sm + kTileBytes + kWBytes);
    uint64_t* mbar = reinterpret_cast<uint64_t*>(sm + kBarOff);
    uint32_t* tslot = reinterpret_cast<uint32_t*>(mbar + 1);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;

    // parameters: W2 into the B operand layout, the narrow layers as fp32
    const __nv_bfloat16* W1 = w;
    const __nv_bfloat16* b1 = W1 + H * 4;
    const __nv_bfloat16* W2 = b1 + H;
    const __nv_bfloat16* b2 = W2 + H * H;
    const __nv_bfloat16* W3 = b2 + H;
    for (int k = tid; k < H * H; k += blockDim.x)
        *reinterpret_cast<__nv_bfloat16*>(B + kmajor_off(k / H, k % H)) = W2[k];
    for (int k = tid; k < H * 4; k += blockDim.x) S.W1[k] = __bfloat162float(W1[k]);
    for (int k = tid; k < H; k += blockDim.x) {
        S.b1[k] = __bfloat162float(b1[k]);
        S.b2[k] = __bfloat162float(b2[k]);
        S.W3[k] = __bfloat162float(W3[k]);
    }
    if (tid == 0) {
        S.b3 = __bfloat162float(W3[H]);
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(mbar)));
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n"
                     ::"r"(smem_u32(tslot)), "r"(kTcCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
    }
    asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
    const uint32_t tmem = *tslot;
    const uint32_t a0 = smem_u32(A), b0 = smem_u32(B);
    uint32_t phase = 0;
    bool ok = true;
    bool drained = true;   // no product is still being written to the accumulator

    for (int64_t base = (int64_t)blockIdx.x * 128; base < n && ok; base += (int64_t)gridDim.x * 128) {
        // layer 1 (fp32) for row tid; relu(z1) as bf16 into the A tile
        int64_t row = base + tid;
        float x[4];
#pragma unroll
        for (int i = 0; i < 4; ++i) x[i] = row < n ? feat[row * 4 + i] : 0.f;
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            uint32_t pk[4];
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                float z[2];
#pragma unroll
                for (int h = 0; h < 2; ++h) {
                    int u = 8 * j + 2 * e + h;
                    float s = S.b1[u];
#pragma unroll
                    for (int i = 0; i < 4; ++i) s += S.W1[u * 4 + i] * x[i];
                    z[h] = fmaxf(s, 0.f);
                }
                pk[e] = pack2(z[0], z[1]);
            }
            *reinterpret_cast<uint4*>(A + kmajor_off(tid, 8 * j)) = make_uint4(pk[0], pk[1], pk[2], pk[3]);
        }
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        __syncthreads();
        if (tid == 0) {
            asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
#pragma unroll
            for (uint32_t s = 0; s < 4; ++s) {
                uint64_t ad = smem_desc(a0 + 256u * s, 128u, 1024u);
                uint64_t bd = smem_desc(b0 + 256u * s, 128u, 1024u);
                asm volatile(
                    "{\n.reg .pred p;\nsetp.ne.b32 p, %4, 0;\n"
                    "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
                    ::"r"(tmem), "l"(ad), "l"(bd), "r"(kTcIdesc), "r"(s));
            }
            asm volatile(
                "tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n"
                ::"r"(smem_u32(mbar)) : "memory");
        }
        // wait for the products (bounded; the whole CTA gives up together)
        if (__syncthreads_or(!wait_phase(mbar, phase))) {
            ok = false;
            // once more (bounded) for the products in flight; if they still
            // have not arrived the accumulator may be in use, so it is not
            // freed (flag 2: the network's tensor-core path is unusable)
            drained = !__syncthreads_or(!wait_phase(mbar, phase));
            if (tid == 0) atomicMax(err, drained ? 1 : 2);
            break;
        }
        phase ^= 1u;
        asm volatile("tcgen05.fence::after_thread_sync;\n" ::: "memory");
        // this warp's 32 accumulator rows: lane = row, 64 columns
        float acc[64];
        uint32_t taddr = tmem + ((uint32_t)(32 * warp) << 16);
#pragma unroll
        for (int c = 0; c < 4; ++c) {
            uint32_t* r = reinterpret_cast<uint32_t*>(acc + 16 * c);
            asm volatile(
                "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,"
                "%12,%13,%14,%15}, [%16];\n"
                : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]),
                  "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]),
                  "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
                : "r"(taddr + 16u * c));
        }
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        // bias, relu, layer 3 (fp32)
        float o = S.b3;
#pragma unroll
        for (int u = 0; u < 64; ++u) o += S.W3[u] * fmaxf(acc[u] + S.b2[u], 0.f);
        int64_t r = base + 32 * warp + lane;
        if (r < n) out[r] = o;
        asm volatile("tcgen05.fence::before_thread_sync;\n" ::: "memory");
        __syncthreads();   // the A tile and the accumulator are free again
    }
    __syncthreads();
    if (warp == 0 && drained)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(tmem),
                     "r"(kTcCols));
}

constexpr size_t kTcSmem = kBarOff + 16;   // + the mbarrier and the TMEM address slot

// Gradient of L = sum_s w_s (out_s - y_s)^2 / sum_s w_s, accumulated into
// grad (fp32, parameter layout) and the loss into *loss.  inv_wsum = 1 /
// sum_s w_s (computed by k_weight_sum).
__global__ void __launch_bounds__(256) k_mlp_grad(const __nv_bfloat16* __restrict__ w,
                                                  const float* __restrict__ feat,
                                                  const float* __restrict__ y,
                                                  const float* __restrict__ wt, int64_t n,
                                                  const float* __restrict__ inv_wsum,
                                                  float* __restrict__ grad,
                                                  float* __restrict__ loss) {
    extern __shared__ __align__(16) unsigned char smem[];
    GradSmem& G = *reinterpret_cast<GradSmem*>(smem);
    SmemNet& S = G.net;
    float *gW1 = G.gW1, *gb1 = G.gb1, *gW2 = G.gW2, *gb2 = G.gb2, *gW3 = G.gW3;
    float& gb3 = G.gb3;
    float& lsum = G.lsum;
    load_net(S, w);
    for (int k = threadIdx.x; k < H * H; k += blockDim.x) gW2[k] = 0.f;
    for (int k = threadIdx.x; k < H * 4; k += blockDim.x) gW1[k] = 0.f;
    for (int k = threadIdx.x; k < H; k += blockDim.x) gb1[k] = gb2[k] = gW3[k] = 0.f;
    if (threadIdx.x == 0) gb3 = lsum = 0.f;
    __syncthreads();
    float iw = *inv_wsum;
    int lane = threadIdx.x & 31, g = lane >> 2, t = lane & 3, wid = threadIdx.x >> 5;
    __nv_bfloat16* dz2T = G.stage[wid][0];   // [unit][sample]
    __nv_bfloat16* h1T = G.stage[wid][1];    // [unit][sample]
    int64_t warp = ((int64_t)blockIdx.x * blockDim.x + threadIdx.x) >> 5;
    int64_t nw = ((int64_t)gridDim.x * blockDim.x) >> 5;
    for (int64_t base = warp * 16; base < n; base += nw * 16) {
        Tile16 T;
        load_features(feat, n, base, T);
        forward16(S, T);
        // dL/dout per row (0 for padding rows)
        float dout[2];
#pragma unroll
        for (int r = 0; r < 2; ++r) {
            int64_t s = base + g + 8 * r;
            float e = s < n ? T.out[r] - y[s] : 0.f;
            float ws = s < n ? wt[s] : 0.f;
            dout[r] = 2.f * ws * e * iw;
            if (t == 0) atomicAdd(&lsum, ws * e * e * iw);
        }
        // dz2 = dout W3 relu'(z2)
        float dz2[8][4];
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int u = 8 * j + 2 * t + (e & 1);
                dz2[j][e] = T.z2[j][e] > 0.f ? dout[e >> 1] * S.W3[u] : 0.f;
            }
        // reduce dW3, db2 over the 16 rows (lanes with equal t share units)
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                float gw3 = dout[0] * fmaxf(T.z2[j][c], 0.f) + dout[1] * fmaxf(T.z2[j][2 + c], 0.f);
                float gbb = dz2[j][c] + dz2[j][2 + c];
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {
                    gw3 += __shfl_xor_sync(kAll, gw3, o);
                    gbb += __shfl_xor_sync(kAll, gbb, o);
                }
                if (g == 0) {
                    atomicAdd(&gW3[8 * j + 2 * t + c], gw3);
                    atomicAdd(&gb2[8 * j + 2 * t + c], gbb);
                }
            }
        {
            float db3 = (t == 0) ? dout[0] + dout[1] : 0.f;
#pragma unroll
            for (int o = 1; o < 32; o <<= 1) db3 += __shfl_xor_sync(kAll, db3, o);
            if (lane == 0) atomicAdd(&gb3, db3);
        }
        // stage dz2^T and relu(z1)^T (bf16) for the dW2 product
#pragma unroll
        for (int j = 0; j < 8; ++j)
#pragma unroll
            for (int e = 0; e < 4; ++e) {
                int u = 8 * j + 2 * t + (e & 1);
                int row = g + 8 * (e >> 1);
                dz2T[u * 16 + row] = __float2bfloat16_rn(dz2[j][e]);
                h1T[u * 16 + row] = __float2bfloat16_rn(fmaxf(T.z1[j][e], 0.f));
            }
        __syncwarp();
        // dW2 = dz2^T (64 x 16) x h1 (16 x 64) on the tensor cores
#pragma unroll
        for (int mt = 0; mt < 4; ++mt) {
            uint32_t a[4];
            const uint32_t* dz = reinterpret_cast<const uint32_t*>(dz2T);
            a[0] = dz[((16 * mt + g) * 16 + 2 * t) >> 1];
            a[1] = dz[((16 * mt + g + 8) * 16 + 2 * t) >> 1];
            a[2] = dz[((16 * mt + g) * 16 + 2 * t + 8) >> 1];
            a[3] = dz[((16 * mt + g + 8) * 16 + 2 * t + 8) >> 1];
            const uint32_t* hh = reinterpret_cast<const uint32_t*>(h1T);
#pragma unroll
            for (int j = 0; j < 8; ++j) {
                float d[4] = {0.f, 0.f, 0.f, 0.f};
                uint32_t b0 = hh[((8 * j + g) * 16 + 2 * t) >> 1];
                uint32_t b1 = hh[((8 * j + g) * 16 + 2 * t + 8) >> 1];
                mma16816(d, a, b0, b1);
                int o0 = 16 * mt + g, i0 = 8 * j + 2 * t;
                atomicAdd(&gW2[o0 * H + i0], d[0]);
                atomicAdd(&gW2[o0 * H + i0 + 1], d[1]);
                atomicAdd(&gW2[(o0 + 8) * H + i0], d[2]);
                atomicAdd(&gW2[(o0 + 8) * H + i0 + 1], d[3]);
            }
        }
        // dh1 = dz2 (16 x 64) x W2 (64 x 64) on the tensor cores; A from the
        // dz2 accumulator tiles, B from W2^T
        uint32_t a2[4][4];
#pragma unroll
        for (int kk = 0; kk < 4; ++kk) {
            const float* lo = dz2[2 * kk];
            const float* hi = dz2[2 * kk + 1];
            a2[kk][0] = pack2(lo[0], lo[1]);
            a2[kk][1] = pack2(lo[2], lo[3]);
            a2[kk][2] = pack2(hi[0], hi[1]);
            a2[kk][3] = pack2(hi[2], hi[3]);
        }
#pragma unroll
        for (int j = 0; j < 8; ++j) {
            float d[4] = {0.f, 0.f, 0.f, 0.f};
            const uint32_t* wt2 = reinterpret_cast<const uint32_t*>(S.W2T + (8 * j + g) * H);
#pragma unroll
            for (int kk = 0; kk < 4; ++kk) mma16816(d, a2[kk], wt2[8 * kk + t], wt2[8 * kk + 4 + t]);
            // dz1 = dh1 relu'(z1); dW1 = dz1 x, db1 = dz1, summed over rows
#pragma unroll
            for (int c = 0; c < 2; ++c) {
                int u = 8 * j + 2 * t + c;
                float d0 = T.z1[j][c] > 0.f ? d[c] : 0.f;
                float d1 = T.z1[j][2 + c] > 0.f ? d[2 + c] : 0.f;
                float gb = d0 + d1;
                float gw[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) gw[i] = d0 * T.x[0][i] + d1 * T.x[1][i];
#pragma unroll
                for (int o = 4; o < 32; o <<= 1) {
                    gb += __shfl_xor_sync(kAll, gb, o);
#pragma unroll
                    for (int i = 0; i < 4; ++i) gw[i] += __shfl_xor_sync(kAll, gw[i], o);
                }
                if (g == 0) {
                    atomicAdd(&gb1[u], gb);
#pragma unroll
                    for (int i = 0; i < 4; ++i) atomicAdd(&gW1[u * 4 + i], gw[i]);
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();
    float* gW1g = grad;
    float* gb1g = gW1g + H * 4;
    float* gW2g = gb1g + H;
    float* gb2g = gW2g + H * H;
    float* gW3g = gb2g + H;
    float* gb3g = gW3g + H;
    for (int k = threadIdx.x; k < H * H; k += blockDim.x) atomicAdd(&gW2g[k], gW2[k]);
    for (int k = threadIdx.x; k < H * 4; k += blockDim.x) atomicAdd(&gW1g[k], gW1[k]);
    for (int k = threadIdx.x; k < H; k += blockDim.x) {
        atomicAdd(&gb1g[k], gb1[k]);
        atomicAdd(&gb2g[k], gb2[k]);
        atomicAdd(&gW3g[k], gW3[k]);
    }
    if (threadIdx.x == 0) {
        atomicAdd(gb3g, gb3);
        atomicAdd(loss, lsum);
    }
}

// 1 / sum of the sample weights (one block).
__global__ void __launch_bounds__(1024) k_weight_sum(const float* __restrict__ wt, int64_t n,
                                                     float* __restrict__ inv) {
    __shared__ float part[32];
    float s = 0.f;
    for (int64_t k = threadIdx.x; k < n; k += blockDim.x) s += wt[k];
    for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kAll, s, o);
    if ((threadIdx.x & 31) == 0) part[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        s = threadIdx.x < (blockDim.x >> 5) ? part[threadIdx.x] : 0.f;
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(kAll, s, o);
        if (threadIdx.x == 0) *inv = s > 0.f ? 1.f / s : 0.f;
    }
}

// Adam step on the fp32 master parameters; refreshes the BF16 copy and
// clears the gradient.
__global__ void k_adam(float* __restrict__ p, float* __restrict__ m, float* __restrict__ v,
                       float* __restrict__ grad, __nv_bfloat16* __restrict__ w, int n, float lr,
                       float b1, float b2, float eps, float c1, float c2) {
    for (int k = blockIdx.x * blockDim.x + threadIdx.x; k < n; k += gridDim.x * blockDim.x) {
        float gk = grad[k];
        float mk = b1 * m[k] + (1.f - b1) * gk;
        float vk = b2 * v[k] + (1.f - b2) * gk * gk;
        m[k] = mk;
        v[k] = vk;
        float pk = p[k] - lr * (mk * c1) / (sqrtf(vk * c2) + eps);
        p[k] = pk;
        w[k] = __float2bfloat16_rn(pk);
        grad[k] = 0.f;
    }
}

// Network features of mesh cell (cell, energy bin) of a geometry: the cell
// centre and the bin's logarithmic centre, shifted and scaled.
__global__ void k_mesh_features(MeshSpec M, float* __restrict__ feat) {
    int64_t n = (int64_t)M.n_cells * M.n_bins;
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        int32_t cell = (int32_t)(k / M.n_bins), b = (int32_t)(k % M.n_bins);
        double x = 0.0, y = 0.0, z = 0.0;
        const gbmc_geometry& g = M.g;
        if (g.kind == GBMC_GEOM_SLAB) {
            x = ((double)cell + 0.5) * g.layer_dx;
        } else if (g.kind == GBMC_GEOM_LATTICE) {
            x = ((double)(cell % g.n) + 0.5) * g.pitch;
            y = ((double)(cell / g.n) + 0.5) * g.pitch;
            z = 0.5 * g.height;
        }
        double le = 0.5 * (log(M.edges[b]) + log(M.edges[b + 1]));
        double raw[4] = {x, y, z, le};
        for (int i = 0; i < 4; ++i) feat[k * 4 + i] = (float)((raw[i] - M.offset[i]) * M.scale[i]);
    }
}

// Window lower bounds from the network's log-importance on the mesh:
// w_lower = C / exp(out), with C set so that the survival weight of the
// source cell / bin is 1 (the source's unit weight sits in its window).
__global__ void k_windows(const float* __restrict__ out, int64_t n, int64_t src,
                          double survival, double* __restrict__ lower) {
    double lc = (double)out[src];
    for (int64_t k = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; k < n;
         k += (int64_t)gridDim.x * blockDim.x) {
        double l = exp(lc - (double)out[k]) / survival;
        if (!(l < 1e300)) l = 1e300;
        if (!(l > 1e-300)) l = 1e-300;
        lower[k] = l;
    }
}

}  // namespace

cudaError_t mlp_forward(const __nv_bfloat16* w, const float* feat, int64_t n, float* out,
                        int* err, int sms, cudaStream_t s) {
    if (n <= 0) return cudaSuccess;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_forward_tc,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)kTcSmem);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    // at most 4 CTAs (4 x 64 TMEM columns) per SM
    int64_t tiles = (n + 127) / 128;
    int blocks = (int)std::min<int64_t>(tiles, (int64_t)sms * 4);
    k_mlp_forward_tc<<<blocks, 128, kTcSmem, s>>>(w, feat, n, out, err);
    return cudaGetLastError();
}

cudaError_t mlp_grad(const __nv_bfloat16* w, const float* feat, const float* y, const float* wt,
                     int64_t n, float* scratch_inv, float* grad, float* loss, int sms,
                     cudaStream_t s) {
    k_weight_sum<<<1, 1024, 0, s>>>(wt, n, scratch_inv);
    int64_t warps = (n + 15) / 16;
    int blocks = (int)std::min<int64_t>((warps + kWarps - 1) / kWarps, (int64_t)sms * 2);
    if (blocks < 1) blocks = 1;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(k_mlp_grad, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)sizeof(GradSmem));
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    k_mlp_grad<<<blocks, 32 * kWarps, sizeof(GradSmem), s>>>(w, feat, y, wt, n, scratch_inv, grad,
                                                             loss);
    return cudaGetLastError();
}

cudaError_t mlp_adam(float* p, float* m, float* v, float* grad, __nv_bfloat16* w, int n, float lr,
                     int step, cudaStream_t s) {
    const float b1 = 0.9f, b2 = 0.999f, eps = 1e-8f;
    float c1 = 1.f / (1.f - powf(b1, (float)step));
    float c2 = 1.f / (1.f - powf(b2, (float)step));
    k_adam<<<(n + 255) / 256, 256, 0, s>>>(p, m, v, grad, w, n, lr, b1, b2, eps, c1, c2);
    return cudaGetLastError();
}

cudaError_t mesh_features(const MeshSpec& M, float* feat, int sms, cudaStream_t s) {
    int64_t n = (int64_t)M.n_cells * M.n_bins;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 4);
    if (blocks < 1) blocks = 1;
    k_mesh_features<<<blocks, 256, 0, s>>>(M, feat);
    return cudaGetLastError();
}

cudaError_t mesh_windows(const MeshSpec& M, const __nv_bfloat16* w, float* feat, float* out,
                         double survival, int64_t src, double* lower, int* err, int sms,
                         cudaStream_t s) {
    int64_t n = (int64_t)M.n_cells * M.n_bins;
    int blocks = (int)std::min<int64_t>((n + 255) / 256, (int64_t)sms * 4);
    k_mesh_features<<<blocks, 256, 0, s>>>(M, feat);
    cudaError_t e = mlp_forward(w, feat, n, out, err, sms, s);
    if (e != cudaSuccess) return e;
    k_windows<<<blocks, 256, 0, s>>>(out, n, src, survival, lower);
    return cudaGetLastError();
}

}  // namespace gbmc
