// Fused inference of the learned tiDAS kernel generator on tcgen05: all four
// layers of the 4 -> 256 -> 256 -> 256 -> n_out MLP (n_out = 64 for a row
// kernel, kz * 64 for a band patch) for a tile of 128 samples, without
// writing hidden activations to global memory.
//
// Persistent: one CTA per SM walks 128-row tiles, two at a time.  Per tile
// the epilogue warps encode the samples into the first layer's operand, and
// after each layer read the FP32 accumulator from tensor memory, add the
// bias, apply ReLU and write the BF16 activations back into shared memory
// (128-byte swizzled, K-major: the next layer's A operand).  The two tiles of
// a round have their own operands and accumulators and take the layers in
// turn (layer l of tile 0, layer l of tile 1, layer l + 1 of tile 0, ...), so
// one tile's epilogue runs while the other's MMAs do.  The weights, identical
// for every tile, stream from L2 by TMA in 64-column chunks through a ring,
// in the order the MMAs consume them.  Roles: warp 0 loads weights (and owns tensor
// memory), warp 1 issues the MMAs, warps 2-5 run encode and epilogues (one
// accumulator row per thread).  The last layer runs in output chunks of up to
// 256 columns, each in the tile's accumulator columns, drained by the
// epilogue before the next chunk's MMAs; its output is scaled per row (the
// apodization sum) and stored in FP32.
#include "common.cuh"
#include "sm103_primitives.cuh"

namespace tidas {
using namespace sm103;

__device__ int g_mlp_infer_wait_error = 0;

int read_clear_mlp_infer_wait_flag(int* v) {
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(v, g_mlp_infer_wait_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_mlp_infer_wait_error, &zero, sizeof(int));
    return check_cuda(e, "mlp infer wait flag");
}

namespace mi {
constexpr int kM = 128;       // samples per tile (UMMA M)
constexpr int kHid = 256;
constexpr int kIO = 64;       // padded input width; output widths are multiples of it
constexpr int kMaxOut = 512;  // widest output (8 kernel rows of 64)
constexpr int kOC = 256;      // output columns per last-layer chunk (UMMA N)
constexpr int kKC = 64;       // K columns per weight chunk / activation chunk
constexpr int kStages = 2;    // weight chunks in flight
constexpr int kTiles = 2;     // tiles per round (ping-pong)
constexpr int kWBytes = kHid * kKC * 2;   // 32 KB (largest chunk)
constexpr int kABytes = kM * kKC * 2;     // 16 KB per activation chunk
constexpr int kAChunks = kHid / kKC;      // 4
constexpr int kBias = 3 * kHid + kMaxOut;
constexpr size_t kSmem = 1024 + (size_t)kStages * kWBytes + (size_t)kTiles * kAChunks * kABytes +
                         1024 + (size_t)kBias * 4;
static_assert(kSmem <= 227 * 1024, "shared memory");
// Layers of a tile as the MMAs take them: 0 (W1), 1, 2 (W2, W3) and
// 3 .. 2 + noc, the output chunks of W4; a layer past 0 has kAChunks
// K-chunks of weights.
__host__ __device__ constexpr int out_chunks(int no) { return (no + kOC - 1) / kOC; }
}  // namespace mi

struct MlpInferArgs {
    float lo[4], hi[4];
};

__global__ void __launch_bounds__(192, 1)
    mlp_infer_kernel(const __grid_constant__ CUtensorMap w1, const __grid_constant__ CUtensorMap w2,
                     const __grid_constant__ CUtensorMap w3, const __grid_constant__ CUtensorMap w4,
                     const float* __restrict__ b1, const float* __restrict__ b2,
                     const float* __restrict__ b3, const float* __restrict__ b4,
                     const double* __restrict__ samples, int n, MlpInferArgs enc,
                     const float* __restrict__ scale, float* __restrict__ out, int ldo, int no) {
    using namespace mi;
    const int noc = out_chunks(no);    // output chunks of the last layer
    const int nl = 3 + noc;            // layers per tile as the MMAs take them
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = smem_align1024(smem_raw);
    uint8_t* sW = base;                                  // [kStages] weight chunks
    uint8_t* sA = sW + kStages * kWBytes;                // [kTiles][kAChunks] activation chunks
    uint64_t* full = (uint64_t*)(sA + kTiles * kAChunks * kABytes);
    uint64_t* empty = full + kStages;
    uint64_t* a_full = empty + kStages;   // [kTiles] epilogue -> MMA: operand written, accumulator read
    uint64_t* acc_full = a_full + kTiles; // [kTiles] MMA -> epilogue: layer done
    uint64_t* done = acc_full + kTiles;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* s_abort = (volatile int*)(tmem_slot + 1);
    float* s_bias = (float*)((uint8_t*)full + 1024);     // b1 | b2 | b3 | b4

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = (n + kM - 1) / kM;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int b = 0; b < kTiles; ++b) {
            mbar_init(&a_full[b], 4);
            mbar_init(&acc_full[b], 1);
        }
        mbar_init(done, 1);
        *s_abort = 0;
        fence_barrier_init();
        prefetch_tensormap(&w1);
        prefetch_tensormap(&w2);
        prefetch_tensormap(&w3);
        prefetch_tensormap(&w4);
    }
    for (int i = threadIdx.x; i < 3 * kHid + no; i += blockDim.x)
        s_bias[i] = i < kHid ? b1[i] : i < 2 * kHid ? b2[i - kHid] : i < 3 * kHid ? b3[i - 2 * kHid]
                                                                              : b4[i - 3 * kHid];
    if (warp == 0) {
        tmem_alloc(tmem_slot, kTiles * kHid);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ weight chunks by TMA
        if (lane == 0) {
            uint32_t st = 0, ph = 0;
            for (int t = blockIdx.x; t < ntiles && !*s_abort; t += kTiles * gridDim.x) {
                const int nt = (t + (int)gridDim.x < ntiles) ? kTiles : 1;  // tiles this round
                bool stop = false;
                // layer l's chunks for tile 0, then for tile 1 (the MMAs' order)
                for (int l = 0; l < nl && !stop; ++l) {
                    const int kc = l == 0 ? 1 : kAChunks;
                    for (int qi = 0; qi < nt * kc; ++qi) {
                        const int c = qi % kc;  // K-chunk of the layer
                        if (!mbar_wait_or_abort(&empty[st], ph ^ 1u, s_abort, &g_mlp_infer_wait_error,
                                                401)) {
                            stop = true;
                            break;
                        }
                        const CUtensorMap* map = l == 0 ? &w1 : l == 1 ? &w2 : l == 2 ? &w3 : &w4;
                        // rows of the chunk: 256 (W1-W3) or output chunk l - 3 of W4
                        const int r0 = l < 3 ? 0 : kOC * (l - 3);
                        const int rows = l < 3 ? kHid : min(kOC, no);  // every W4 chunk full
                        mbar_arrive_expect_tx(&full[st], (uint32_t)(rows * kKC * 2));
                        asm volatile(
                            "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes"
                            " [%0], [%1, {%2, %3}], [%4];" ::"r"(smem_u32(sW + st * kWBytes)),
                            "l"(reinterpret_cast<uint64_t>(map)), "r"(c * kKC), "r"(r0),
                            "r"(smem_u32(&full[st]))
                            : "memory");
                        if (++st == kStages) { st = 0; ph ^= 1; }
                    }
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------------- MMAs
        if (lane == 0) {
            const uint32_t id_h = idesc_bf16_f32(kM, kHid), id_o = idesc_bf16_f32(kM, min(kOC, no));
            uint32_t st = 0, ph = 0, aph[kTiles] = {0, 0};
            bool ok = true;
            for (int t = blockIdx.x; t < ntiles && ok; t += kTiles * gridDim.x) {
                const int nt = (t + (int)gridDim.x < ntiles) ? kTiles : 1;
                for (int l = 0; l < nl && ok; ++l) {
                    for (int b = 0; b < nt && ok; ++b) {
                        ok = mbar_wait_or_abort(&a_full[b], aph[b], s_abort, &g_mlp_infer_wait_error, 402);
                        aph[b] ^= 1u;
                        if (!ok) break;
                        tc_fence_after();
                        const uint32_t acc = tmem + (uint32_t)(b * kHid);
                        const uint8_t* ab = sA + (size_t)b * kAChunks * kABytes;
                        const int nchunks = l == 0 ? 1 : kAChunks;
                        for (int c = 0; c < nchunks; ++c) {
                            ok = mbar_wait_or_abort(&full[st], ph, s_abort, &g_mlp_infer_wait_error, 403);
                            if (!ok) break;
                            tc_fence_after();
                            const uint32_t a = smem_u32(ab + c * kABytes), w = smem_u32(sW + st * kWBytes);
#pragma unroll
                            for (int kk = 0; kk < kKC / 16; ++kk)
                                mma_f16(acc, desc_sw128_kmajor(a) + 2 * kk, desc_sw128_kmajor(w) + 2 * kk,
                                        l >= 3 ? id_o : id_h, (c > 0 || kk > 0) ? 1u : 0u);
                            mma_commit(&empty[st]);
                            if (++st == kStages) { st = 0; ph ^= 1; }
                        }
                        if (ok) mma_commit(&acc_full[b]);
                    }
                }
            }
            mma_commit(done);
            mbar_wait(done, 0, &g_mlp_infer_wait_error, 404);  // MMAs in flight end before dealloc
        }
        __syncwarp();
    } else {
        // ------------------------------------ encode and epilogues, one row each
        const int q4 = warp & 3;                          // tensor-memory lane quadrant
        const int r = 32 * q4 + lane;                     // row of the tile
        const uint32_t lane_base = (uint32_t)(32 * q4) << 16;
        const int swz = r & 7;
        uint32_t cph[kTiles] = {0, 0};
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += kTiles * gridDim.x) {
            const int nt = (t + (int)gridDim.x < ntiles) ? kTiles : 1;
            // encode: four features in [-1, 1], zeros in columns 4..63
            for (int b = 0; b < nt; ++b) {
                const int row = (t + b * (int)gridDim.x) * kM + r;
                uint8_t* const arow = sA + (size_t)b * kAChunks * kABytes + (r >> 3) * 1024 + (r & 7) * 128;
                uint4 v = make_uint4(0, 0, 0, 0);
                if (row < n) {
                    float f[4];
#pragma unroll
                    for (int k = 0; k < 4; ++k)
                        f[k] = 2.f * ((float)samples[(size_t)row * 4 + k] - enc.lo[k]) /
                                   (enc.hi[k] - enc.lo[k]) - 1.f;
                    const __nv_bfloat162 p0 = __floats2bfloat162_rn(f[0], f[1]);
                    const __nv_bfloat162 p1 = __floats2bfloat162_rn(f[2], f[3]);
                    v.x = *reinterpret_cast<const uint32_t*>(&p0);
                    v.y = *reinterpret_cast<const uint32_t*>(&p1);
                }
                *reinterpret_cast<uint4*>(arow + ((0 ^ swz) << 4)) = v;
#pragma unroll
                for (int u = 1; u < 8; ++u)
                    *reinterpret_cast<uint4*>(arow + ((u ^ swz) << 4)) = make_uint4(0, 0, 0, 0);
                fence_proxy_async_smem();
                tc_fence_before();
                __syncwarp();
                if (lane == 0) mbar_arrive(&a_full[b]);
            }
            for (int l = 0; l < nl && ok; ++l) {
                for (int b = 0; b < nt && ok; ++b) {
                    const int row = (t + b * (int)gridDim.x) * kM + r;
                    uint8_t* const arow = sA + (size_t)b * kAChunks * kABytes + (r >> 3) * 1024 + (r & 7) * 128;
                    const uint32_t acc_col = (uint32_t)(b * kHid);
                    ok = mbar_wait_or_abort(&acc_full[b], cph[b], s_abort, &g_mlp_infer_wait_error, 405);
                    cph[b] ^= 1u;
                    if (!ok) break;
                    tc_fence_after();
                    if (l < 3) {
                        // bias, ReLU, BF16 into the next layer's operand
                        const float* bl = s_bias + l * kHid;
#pragma unroll 1
                        for (int j = 0; j < kHid; j += 32) {
                            uint32_t acc[32];
                            tmem_ld_32x32b_x32(tmem + lane_base + acc_col + (uint32_t)j, acc);
                            tmem_ld_wait();
                            uint32_t pk[16];
#pragma unroll
                            for (int e = 0; e < 16; ++e) {
                                const float x0 = fmaxf(__uint_as_float(acc[2 * e]) + bl[j + 2 * e], 0.f);
                                const float x1 = fmaxf(__uint_as_float(acc[2 * e + 1]) + bl[j + 2 * e + 1], 0.f);
                                const __nv_bfloat162 p = __floats2bfloat162_rn(x0, x1);
                                pk[e] = *reinterpret_cast<const uint32_t*>(&p);
                            }
                            uint8_t* chunk = arow + (j / kKC) * kABytes;
#pragma unroll
                            for (int u = 0; u < 4; ++u) {
                                const int unit = ((j % kKC) >> 3) + u;
                                *reinterpret_cast<uint4*>(chunk + ((unit ^ swz) << 4)) =
                                    make_uint4(pk[4 * u], pk[4 * u + 1], pk[4 * u + 2], pk[4 * u + 3]);
                            }
                        }
                        fence_proxy_async_smem();
                        tc_fence_before();
                        __syncwarp();
                        if (lane == 0) mbar_arrive(&a_full[b]);
                    } else {
                        // output chunk l - 3: bias, apodization scale, FP32 store
                        const int o0 = kOC * (l - 3), ow = min(kOC, no);
                        const float* bl = s_bias + 3 * kHid + o0;
                        const float sc = (row < n && scale) ? scale[row] : 1.f;
#pragma unroll 1
                        for (int j = 0; j < ow; j += 32) {
                            uint32_t acc[32];
                            tmem_ld_32x32b_x32(tmem + lane_base + acc_col + (uint32_t)j, acc);
                            tmem_ld_wait();
                            if (row < n) {
                                float4* dst = reinterpret_cast<float4*>(out + (size_t)row * ldo + o0 + j);
#pragma unroll
                                for (int e = 0; e < 32; e += 4)
                                    dst[e / 4] = make_float4((__uint_as_float(acc[e]) + bl[j + e]) * sc,
                                                             (__uint_as_float(acc[e + 1]) + bl[j + e + 1]) * sc,
                                                             (__uint_as_float(acc[e + 2]) + bl[j + e + 2]) * sc,
                                                             (__uint_as_float(acc[e + 3]) + bl[j + e + 3]) * sc);
                            }
                        }
                        tc_fence_before();
                        if (l + 1 < nl) {
                            // accumulator drained: the next output chunk may start
                            __syncwarp();
                            if (lane == 0) mbar_arrive(&a_full[b]);
                        }
                        // after the last chunk, the next round's encode overwrites
                        // this tile's operand only after its last MMAs, which
                        // acc_full saw complete
                    }
                }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, kTiles * kHid);
    }
}

int make_map_2d_bf16(CUtensorMap* map, const void* ptr, int rows, int cols, int box_rows);
int sm_count();

int launch_mlp_infer(const double* samples, int n, const float* lo4, const float* hi4,
                     const void* const* w16, const float* const* bias, const float* scale,
                     float* out, int ldo, int no, cudaStream_t st) {
    using namespace mi;
    CUtensorMap m[4];
    const int rows[4] = {kHid, kHid, kHid, no}, cols[4] = {kIO, kHid, kHid, kHid};
    const int box[4] = {kHid, kHid, kHid, no < kOC ? no : kOC};
    for (int l = 0; l < 4; ++l) {
        int rc = make_map_2d_bf16(&m[l], w16[l], rows[l], cols[l], box[l]);
        if (rc) return rc;
    }
    MlpInferArgs enc;
    for (int k = 0; k < 4; ++k) {
        enc.lo[k] = lo4[k];
        enc.hi[k] = hi4[k];
    }
    TIDAS_CUDA(cudaFuncSetAttribute(mlp_infer_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)kSmem));
    const int ntiles = (n + kM - 1) / kM;
    const int grid = ntiles < sm_count() ? ntiles : sm_count();
    mlp_infer_kernel<<<grid, 192, kSmem, st>>>(m[0], m[1], m[2], m[3], bias[0], bias[1], bias[2],
                                               bias[3], samples, n, enc, scale, out, ldo, no);
    return check_launch("mlp_infer_kernel");
}

}  // namespace tidas

using namespace tidas;

extern "C" int tidas_mlp_infer(const double* samples, int64_t n, const float* lo4, const float* hi4,
                               const void* const* w16, const float* const* bias, const float* scale,
                               float* out, int32_t ldo, int32_t n_out, void* stream) {
    TIDAS_REQUIRE(samples && lo4 && hi4 && w16 && bias && out, "tidas_mlp_infer: null pointer");
    TIDAS_REQUIRE(n >= 1 && n <= 0x7fffffff, "tidas_mlp_infer: bad n");
    TIDAS_REQUIRE(n_out >= 64 && n_out % 64 == 0 && n_out <= mi::kMaxOut &&
                      (n_out <= mi::kOC || n_out % mi::kOC == 0),
                  "tidas_mlp_infer: n_out must be 64, 128, 192, 256 or 512 (got %d)", n_out);
    TIDAS_REQUIRE(ldo >= n_out && ldo % 4 == 0 && ((uintptr_t)out % 16) == 0,
                  "tidas_mlp_infer: out needs ldo >= n_out, ldo %% 4 == 0 and 16-byte alignment");
    for (int l = 0; l < 4; ++l)
        TIDAS_REQUIRE(w16[l] && bias[l] && ((uintptr_t)w16[l] % 16) == 0,
                      "tidas_mlp_infer: layer %d weights / bias missing or misaligned", l);
    return launch_mlp_infer(samples, (int)n, lo4, hi4, w16, bias, scale, out, ldo, n_out,
                            (cudaStream_t)stream);
}
