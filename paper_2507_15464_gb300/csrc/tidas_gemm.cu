// tiDAS (Eq. (2.13)) as per-row Toeplitz GEMMs on the tcgen05 tensor cores.
//
// For one image row z the lateral convolution of every frame is
//     Y[f, x] = sum_j R[f, j] * T_z[j, x],   T_z[j, x] = h_z[x - j + c],
// a dense contraction over the band |x - j| <= 32 of a Toeplitz matrix.
// Work item = (row z, 128 frames, 2 output tiles of 128 columns): UMMA
// M = 128 frames, N = 128 columns, K = the input columns the tiles read,
// [128 s - 32, 128 s + 160) for tile s, in chunks of 64 columns (the
// 128-byte swizzle width of BF16).  T_z restricted to (chunk offset c',
// tile) does not depend on the tile (shift invariance): three 128 x 64
// operand tiles per row, built in shared memory from the row's taps, serve
// every tile of the row.
//
// Persistent, warp-specialised kernel; each CTA walks a contiguous range of
// items (consecutive items share a row):
//   warp 0      TMA producer of BF16 input chunks (zero fill outside the row)
//   warp 1      tensor-memory owner; lane 0 issues the MMAs
//   warps 2-5   epilogue: tensor memory -> registers -> swizzled shared tile
//               -> TMA tensor store (whole 128-byte lines)
//   warps 6-7   build the next row's Toeplitz tiles (double buffered)
//   warps 8-11  (residual variant) load FP32 input and split it into BF16
//               hi / lo operand tiles
// Accumulators are double buffered in tensor memory so the epilogue of one
// item overlaps the MMAs of the next.  The residual variant adds the two
// first-order low-part products of r = r_hi + r_lo, h = h_hi + h_lo (r_lo,
// h_lo the BF16 roundings of the remainders) into the same accumulators.
#include "common.cuh"
#include "sm103_primitives.cuh"

namespace tidas {
// Written by bounded waits of the tensor-core kernels; read by tidas_device_status.
__device__ int g_wait_error = 0;

using namespace sm103;

namespace gemm {
constexpr int kM = 128;                    // frames per item (UMMA M)
constexpr int kN = 128;                    // outputs per tile (UMMA N)
constexpr int kKC = 64;                    // input columns per K-chunk
constexpr int kTilesPerItem = 2;
constexpr int kChunkBytes = kM * kKC * 2;  // 16 KB of BF16
constexpr int kBTileBytes = kN * kKC * 2;  // 16 KB
constexpr int kOutTileBytes = 32 * 32 * 4; // 32 frames x 32 columns of FP32
constexpr uint32_t kAccCols = kTilesPerItem * kN;  // 256 columns per accumulator buffer
constexpr uint32_t kTmemCols = 2 * kAccCols;       // double buffered
constexpr uint32_t kIdesc = idesc_bf16_f32(kM, kN);
constexpr int kWaitEmpty = 101, kWaitFull = 102, kWaitAcc = 103, kWaitDrain = 104, kWaitConv = 105,
              kWaitB = 106, kWaitAccFree = 107;

template <bool RESID>
struct Cfg {
    static constexpr int kStages = RESID ? 2 : 4;   // operand ring (BF16 hi[/lo] tiles)
    static constexpr int kBBufs = RESID ? 1 : 2;
    static constexpr int kBParts = RESID ? 2 : 1;   // hi [, lo]
    static constexpr int kAParts = RESID ? 2 : 1;
    static constexpr int kWarps = RESID ? 12 : 8;
    static constexpr int kThreads = kWarps * 32;
    static constexpr size_t kOffA = 0;
    static constexpr size_t kOffB = kOffA + (size_t)kStages * kAParts * kChunkBytes;
    static constexpr size_t kOffO = kOffB + (size_t)kBBufs * kBParts * 3 * kBTileBytes;
    static constexpr size_t kOffBar = kOffO + (size_t)4 * 2 * kOutTileBytes;
    static constexpr size_t kSmem = 1024 + kOffBar + 1024;  // barriers, TMEM slot, taps
};

struct Item {
    int z, m0, s0, s1;
};
__device__ __forceinline__ Item decode(int it, int nh, int nm, int ntiles) {
    Item r;
    const int h = it % nh;
    r.m0 = ((it / nh) % nm) * kM;
    r.z = it / (nh * nm);
    r.s0 = h * kTilesPerItem;
    r.s1 = min(ntiles, r.s0 + kTilesPerItem);
    return r;
}
}  // namespace gemm

template <bool RESID>
__global__ void __launch_bounds__(gemm::Cfg<RESID>::kThreads, 1)
    tidas_gemm_kernel(const __grid_constant__ CUtensorMap tmap_in,
                      const __grid_constant__ CUtensorMap tmap_out, const float* __restrict__ in32,
                      const float* __restrict__ kern, int taps, int center, int adjoint, int nz,
                      int nx, int nf) {
    using namespace gemm;
    using C = Cfg<RESID>;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = smem_align1024(smem_raw);
    uint8_t* sA = base + C::kOffA;  // [stage][part] BF16 tiles
    uint8_t* sB = base + C::kOffB;  // [buf][part][3] Toeplitz tiles
    uint8_t* sO = base + C::kOffO;  // [epilogue warp][2] output staging tiles
    uint64_t* full = (uint64_t*)(base + C::kOffBar);
    uint64_t* empty = full + C::kStages;
    uint64_t* b_full = empty + C::kStages;
    uint64_t* b_empty = b_full + 2;
    uint64_t* acc_full = b_empty + 2;
    uint64_t* acc_empty = acc_full + 2;
    uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);
    volatile int* s_abort = (volatile int*)(tmem_slot + 1);
    float* s_taps = (float*)(tmem_slot + 4);  // [kBBufs][64]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int ntiles = (nx + kN - 1) / kN;
    const int nh = (ntiles + kTilesPerItem - 1) / kTilesPerItem;
    const int nm = (nf + kM - 1) / kM;
    const int total = nz * nm * nh;
    const int it_begin = (int)((long long)blockIdx.x * total / gridDim.x);
    const int it_end = (int)((long long)(blockIdx.x + 1) * total / gridDim.x);

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::kStages; ++s) {
            mbar_init(&full[s], RESID ? 4 : 1);  // TMA (tx) or the four converter warps
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&b_full[s], 2);
            mbar_init(&b_empty[s], 1);
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], 4);
        }
        *s_abort = 0;
        fence_barrier_init();
        if (!RESID) prefetch_tensormap(&tmap_in);
        prefetch_tensormap(&tmap_out);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer
        if (!RESID && lane == 0) {
            uint32_t st = 0, ph = 0;
            int issued = 0;
            for (int it = it_begin; it < it_end && !*s_abort; ++it) {
                const Item I = decode(it, nh, nm, ntiles);
                for (int c = 2 * I.s0; c <= 2 * I.s1; ++c) {
                    if (!mbar_wait(&empty[st], ph ^ 1, &g_wait_error, kWaitEmpty)) {
                        *s_abort = 1;
                        break;
                    }
                    mbar_arrive_expect_tx(&full[st], kChunkBytes);
                    tma_load_3d(sA + st * kChunkBytes, &tmap_in, &full[st], kKC * c - 32, I.z,
                                I.m0);
                    if (++st == (uint32_t)C::kStages) { st = 0; ph ^= 1; }
                    ++issued;
                }
            }
            if (*s_abort) {
                // let issued copies land before shared memory is released
                for (int q = 0; q < min(issued, C::kStages); ++q) {
                    st = (st == 0) ? C::kStages - 1 : st - 1;
                    if (st == (uint32_t)C::kStages - 1) ph ^= 1;
                    mbar_wait(&full[st], ph, &g_wait_error, kWaitDrain);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // --------------------------------------------------- MMA issuer
        if (lane == 0) {
            uint32_t st = 0, ph = 0;
            int prev_z = -1, nrow = -1, k = 0;
            for (int it = it_begin; it < it_end && !*s_abort; ++it, ++k) {
                const Item I = decode(it, nh, nm, ntiles);
                if (I.z != prev_z) {
                    if (nrow >= 0) mma_commit(&b_empty[nrow % C::kBBufs]);
                    ++nrow;
                    prev_z = I.z;
                    if (!mbar_wait(&b_full[nrow % C::kBBufs], (nrow / C::kBBufs) & 1,
                                   &g_wait_error, kWaitB)) {
                        *s_abort = 1;
                        break;
                    }
                }
                const int ab = k & 1;
                if (!mbar_wait(&acc_empty[ab], ((k >> 1) & 1) ^ 1, &g_wait_error, kWaitAccFree)) {
                    *s_abort = 1;
                    break;
                }
                tc_fence_after();
                const uint8_t* bt = sB + (size_t)(nrow % C::kBBufs) * C::kBParts * 3 * kBTileBytes;
                for (int c = 2 * I.s0; c <= 2 * I.s1; ++c) {
                    if (!mbar_wait(&full[st], ph, &g_wait_error, kWaitFull)) {
                        *s_abort = 1;
                        break;
                    }
                    tc_fence_after();
                    // descriptors formed once per chunk; a K-step adds 32 bytes (2)
                    const uint64_t da_hi = desc_sw128_kmajor(smem_u32(sA + st * C::kAParts * kChunkBytes));
                    const uint64_t da_lo = da_hi + (uint64_t)(kChunkBytes >> 4);
                    const uint64_t db = desc_sw128_kmajor(smem_u32(bt));
                    // tile tl (absolute) from Toeplitz part cp of this chunk
                    auto tile = [&](int tl, int cp) {
                        const uint32_t d = tmem_base + (uint32_t)(ab * kAccCols) +
                                           (uint32_t)((tl - I.s0) * kN);
                        const uint64_t bh = db + (uint64_t)(cp * (kBTileBytes >> 4));
                        const uint64_t bl = bh + (uint64_t)(3 * (kBTileBytes >> 4));
#pragma unroll
                        for (int kk = 0; kk < kKC / 16; ++kk) {
                            mma_f16(d, da_hi + 2 * kk, bh + 2 * kk, kIdesc,
                                    (cp > 0 || kk > 0) ? 1u : 0u);
                            if (RESID) {
                                mma_f16(d, da_lo + 2 * kk, bh + 2 * kk, kIdesc, 1u);
                                mma_f16(d, da_hi + 2 * kk, bl + 2 * kk, kIdesc, 1u);
                            }
                        }
                    };
                    if ((c & 1) == 0 && c / 2 - 1 >= I.s0) tile(c / 2 - 1, 2);
                    if (c / 2 < I.s1) tile(c / 2, c & 1);
                    mma_commit(&empty[st]);
                    if (++st == (uint32_t)C::kStages) { st = 0; ph ^= 1; }
                }
                mma_commit(&acc_full[ab]);
            }
            if (nrow >= 0) mma_commit(&b_empty[nrow % C::kBBufs]);
        }
        __syncwarp();
    } else if (warp < 6) {
        // ------------------------------------------------------ epilogue
        const int quarter = warp & 3;  // tensor-memory lanes 32*quarter .. +31
        uint8_t* stage_buf = sO + (size_t)(warp - 2) * 2 * kOutTileBytes;
        int k = 0, q = 0;
        for (int it = it_begin; it < it_end && !*s_abort; ++it, ++k) {
            const Item I = decode(it, nh, nm, ntiles);
            const int ab = k & 1;
            if (!mbar_wait(&acc_full[ab], (k >> 1) & 1, &g_wait_error, kWaitAcc)) {
                *s_abort = 1;
                break;
            }
            tc_fence_after();
            for (int s = I.s0; s < I.s1; ++s) {
#pragma unroll 1
                for (int j = 0; j < kN / 32; ++j, ++q) {
                    uint32_t r[32];
                    tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                           (uint32_t)(ab * kAccCols + (s - I.s0) * kN + j * 32),
                                       r);
                    tmem_ld_wait();
                    uint8_t* tile = stage_buf + (q & 1) * kOutTileBytes;
                    // the store issued two tiles ago must have finished reading `tile`
                    if (lane == 0) bulk_wait_read<1>();
                    __syncwarp();
                    // row `lane` of the 32 x 32 tile, 16-byte chunks XOR-swizzled by row
#pragma unroll
                    for (int c4 = 0; c4 < 8; ++c4)
                        *reinterpret_cast<uint4*>(tile + lane * 128 + ((c4 ^ (lane & 7)) << 4)) =
                            make_uint4(r[4 * c4], r[4 * c4 + 1], r[4 * c4 + 2], r[4 * c4 + 3]);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_3d(&tmap_out, tile, s * kN + j * 32, I.z, I.m0 + quarter * 32);
                        bulk_commit();
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ab]);
        }
        if (lane == 0) bulk_wait<0>();
        __syncwarp();
    } else if (warp < 8) {
        // --------------------------------------- Toeplitz operand builders
        const int bt = threadIdx.x - 6 * 32;  // 0..63
        int prev_z = -1, nrow = -1;
        for (int it = it_begin; it < it_end; ++it) {
            const Item I = decode(it, nh, nm, ntiles);
            if (I.z == prev_z) continue;
            prev_z = I.z;
            ++nrow;
            const int b = nrow % C::kBBufs;
            const bool ok = mbar_wait_or_abort(&b_empty[b], ((nrow / C::kBBufs) & 1) ^ 1, s_abort,
                                               &g_wait_error, kWaitB);
            float* tp = s_taps + b * 64;
            if (ok && bt < 64) tp[bt] = bt < taps ? __ldg(kern + (size_t)I.z * taps + bt) : 0.f;
            // the taps are in; leave together if any builder or role gave up
            if (named_bar_or<1>(64, !ok || *s_abort)) break;
            uint8_t* dst = sB + (size_t)b * C::kBParts * 3 * kBTileBytes;
            for (int idx = bt; idx < 3 * kN * kKC / 2; idx += 64) {
                // two consecutive k per thread
                const int c = idx / (kN * kKC / 2), rem = idx % (kN * kKC / 2);
                const int n = rem / (kKC / 2), k2 = (rem % (kKC / 2)) * 2;
                float v[2];
#pragma unroll
                for (int e = 0; e < 2; ++e) {
                    const int kk = k2 + e;
                    const int t = adjoint ? (kk + kKC * c - n - 32 + center)
                                          : (n - kk - kKC * c + 32 + center);
                    v[e] = (t >= 0 && t < taps) ? tp[t] : 0.f;
                }
                const __nv_bfloat162 hi = __floats2bfloat162_rn(v[0], v[1]);
                const uint32_t off = c * kBTileBytes + sw128_offset(n, k2);
                *reinterpret_cast<__nv_bfloat162*>(dst + off) = hi;
                if (RESID) {
                    const float2 hf = __bfloat1622float2(hi);
                    *reinterpret_cast<__nv_bfloat162*>(dst + 3 * kBTileBytes + off) =
                        __floats2bfloat162_rn(v[0] - hf.x, v[1] - hf.y);
                }
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&b_full[b]);
        }
    } else if (RESID) {
        // ------------------------- FP32 input -> BF16 hi / lo operand tiles
        const int ct = threadIdx.x - 8 * 32;  // 0..127
        uint32_t ast = 0, aph = 0;
        for (int it = it_begin; it < it_end && !*s_abort; ++it) {
            const Item I = decode(it, nh, nm, ntiles);
            for (int c = 2 * I.s0; c <= 2 * I.s1; ++c) {
                if (*s_abort || !mbar_wait(&empty[ast], aph ^ 1, &g_wait_error, kWaitConv)) {
                    *s_abort = 1;
                    break;
                }
                uint8_t* dhi = sA + ast * 2 * kChunkBytes;
                uint8_t* dlo = dhi + kChunkBytes;
                const int xb = kKC * c - 32;
                float4 v[16];
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int id = ct + 128 * i;
                    const int row = id >> 4, x = xb + (id & 15) * 4;
                    const int f = I.m0 + row;
                    v[i] = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (f < nf && x >= 0 && x < nx)
                        v[i] = __ldcs(reinterpret_cast<const float4*>(
                            in32 + ((size_t)f * nz + I.z) * nx + x));
                }
                // L2 prefetch of the next chunk (of this item, else the next
                // item's first): row ct of it, its two 128-byte lines
                {
                    int pz = I.z, pm = I.m0, pc = c + 1;
                    bool more = pc <= 2 * I.s1;
                    if (!more && it + 1 < it_end) {
                        const Item J = decode(it + 1, nh, nm, ntiles);
                        pz = J.z;
                        pm = J.m0;
                        pc = 2 * J.s0;
                        more = true;
                    }
                    const int f = pm + ct;
                    if (more && f < nf) {
#pragma unroll
                        for (int h = 0; h < 2; ++h) {
                            const int x = kKC * pc - 32 + 32 * h;
                            if (x >= 0 && x < nx)
                                prefetch_l2(in32 + ((size_t)f * nz + pz) * nx + x);
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < 16; ++i) {
                    const int id = ct + 128 * i;
                    const int row = id >> 4, kq = (id & 15) * 4;
                    const __nv_bfloat162 h01 = __floats2bfloat162_rn(v[i].x, v[i].y);
                    const __nv_bfloat162 h23 = __floats2bfloat162_rn(v[i].z, v[i].w);
                    const float2 f01 = __bfloat1622float2(h01), f23 = __bfloat1622float2(h23);
                    const __nv_bfloat162 l01 = __floats2bfloat162_rn(v[i].x - f01.x, v[i].y - f01.y);
                    const __nv_bfloat162 l23 = __floats2bfloat162_rn(v[i].z - f23.x, v[i].w - f23.y);
                    const uint32_t off = sw128_offset(row, kq);
                    uint2 ph2, pl2;
                    ph2.x = *reinterpret_cast<const uint32_t*>(&h01);
                    ph2.y = *reinterpret_cast<const uint32_t*>(&h23);
                    pl2.x = *reinterpret_cast<const uint32_t*>(&l01);
                    pl2.y = *reinterpret_cast<const uint32_t*>(&l23);
                    *reinterpret_cast<uint2*>(dhi + off) = ph2;
                    *reinterpret_cast<uint2*>(dlo + off) = pl2;
                }
                fence_proxy_async_smem();
                __syncwarp();
                if (lane == 0) mbar_arrive(&full[ast]);
                if (++ast == (uint32_t)C::kStages) { ast = 0; aph ^= 1; }
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

// ------------------------------------------------------------------ host
typedef CUresult (*EncodeTiledFn)(CUtensorMap*, CUtensorMapDataType, cuuint32_t, void*,
                                  const cuuint64_t*, const cuuint64_t*, const cuuint32_t*,
                                  const cuuint32_t*, CUtensorMapInterleave, CUtensorMapSwizzle,
                                  CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiledFn encode_fn() {
    static EncodeTiledFn fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault,
                                             &q) == cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = (EncodeTiledFn)p;
    }
    return fn;
}

// 3D map over a [nf][nz][nx] array; box = box_x columns x 1 row x box_f frames
int make_map_3d(CUtensorMap* map, const void* ptr, CUtensorMapDataType dt, int esize, int nz,
                int nx, int nf, int box_x, int box_f, CUtensorMapSwizzle sw) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(TIDAS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[3] = {(cuuint64_t)nx, (cuuint64_t)nz, (cuuint64_t)nf};
    cuuint64_t strides[2] = {(cuuint64_t)nx * esize, (cuuint64_t)nx * nz * esize};
    cuuint32_t box[3] = {(cuuint32_t)box_x, 1u, (cuuint32_t)box_f};
    cuuint32_t estr[3] = {1u, 1u, 1u};
    CUresult r = enc(map, dt, 3, const_cast<void*>(ptr), dims, strides, box, estr,
                     CU_TENSOR_MAP_INTERLEAVE_NONE, sw, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                     CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(TIDAS_ERR_CUDA, "cuTensorMapEncodeTiled failed (%d)", (int)r);
    return TIDAS_OK;
}

// 2D map over a row-major BF16 [rows][cols] matrix; box = 64 columns x box_rows
// rows, 128-byte swizzle (the K-major UMMA operand layout)
int make_map_2d_bf16(CUtensorMap* map, const void* ptr, int rows, int cols, int box_rows) {
    EncodeTiledFn enc = encode_fn();
    if (!enc) return set_error(TIDAS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
    cuuint64_t dims[2] = {(cuuint64_t)cols, (cuuint64_t)rows};
    cuuint64_t strides[1] = {(cuuint64_t)cols * 2};
    cuuint32_t box[2] = {64u, (cuuint32_t)box_rows};
    cuuint32_t estr[2] = {1u, 1u};
    CUresult r = enc(map, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, const_cast<void*>(ptr), dims, strides,
                     box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_128B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    if (r != CUDA_SUCCESS)
        return set_error(TIDAS_ERR_CUDA, "cuTensorMapEncodeTiled (2D) failed (%d)", (int)r);
    return TIDAS_OK;
}

int sm_count() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0) n = 148;
    }
    return n;
}

int launch_tidas_gemm(const float* kern, int taps, int center, bool adjoint, int nz, int nx,
                      const void* in, float* out, int nf, bool resid, cudaStream_t st) {
    CUtensorMap map_in, map_out;
    // output: 32 columns x 1 row x 32 frames of FP32, 128-byte swizzled staging
    int rc = make_map_3d(&map_out, out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nz, nx, nf, 32, 32,
                         CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    if (resid) {
        map_in = map_out;  // unused by the residual kernel (it reads FP32 directly)
    } else {
        rc = make_map_3d(&map_in, in, CU_TENSOR_MAP_DATA_TYPE_BFLOAT16, 2, nz, nx, nf, gemm::kKC,
                         gemm::kM, CU_TENSOR_MAP_SWIZZLE_128B);
        if (rc) return rc;
    }
    const int ntiles = (nx + gemm::kN - 1) / gemm::kN;
    const int items = nz * ((nf + gemm::kM - 1) / gemm::kM) *
                      ((ntiles + gemm::kTilesPerItem - 1) / gemm::kTilesPerItem);
    const int grid = items < sm_count() ? items : sm_count();
    if (resid) {
        using C = gemm::Cfg<true>;
        TIDAS_CUDA(cudaFuncSetAttribute(tidas_gemm_kernel<true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)C::kSmem));
        tidas_gemm_kernel<true><<<grid, C::kThreads, C::kSmem, st>>>(
            map_in, map_out, (const float*)in, kern, taps, center, adjoint ? 1 : 0, nz, nx, nf);
    } else {
        using C = gemm::Cfg<false>;
        TIDAS_CUDA(cudaFuncSetAttribute(tidas_gemm_kernel<false>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                             (int)C::kSmem));
        tidas_gemm_kernel<false><<<grid, C::kThreads, C::kSmem, st>>>(
            map_in, map_out, nullptr, kern, taps, center, adjoint ? 1 : 0, nz, nx, nf);
    }
    return check_launch("tidas_gemm_kernel");
}

// ------------------------------------------------- 2D band kernels (tcgen05)
// Y_z = sum_u R_{j(u)} T_{j(u), u}: the row-wise Toeplitz GEMM summed over the
// kz input rows j = z - u + kz/2 (adjoint: j = z + u - kz/2, kernel row z)
// into the same accumulators.  A step = (item, u): the producer copies the
// item's input chunks of row j, six builder warps write that step's band
// matrix (double buffered), the MMA warp issues the item's MMAs.
//
// The input is first repacked into the operand's shared-memory image: chunk q
// of (row z, frame tile m) holds columns [64 q - 32, 64 q + 32) of 128 frames
// as a 16 KB 128-byte-swizzled K-major tile, zero outside the grid, so that
// the producer moves two neighbouring chunks (a 32 KB stage) with one
// contiguous bulk copy.  A tiled tensor copy moves a 128-byte row at a time,
// and the issuing thread of the MMAs pays a barrier wait and a commit per
// stage while the tensor pipe, whose queue holds about one MMA, runs dry:
// stages of 2 chunks (3 per step instead of 5) keep it fed.
namespace gemm2 {
constexpr int kStages = 3;
constexpr int kStageBytes = 2 * gemm::kChunkBytes;  // two 64-column chunks
constexpr int kBuilders = 6;  // warps 6 .. 11
constexpr int kMma2Warp = 6 + kBuilders;           // second MMA issuer (tile 1)
constexpr int kThreads = 32 * (kMma2Warp + 1);
// The three Toeplitz tiles of a step (part cp = 0, 1, 2 of a tile's three
// input chunks) are windows of one band matrix G[r][k], r in [-128, 128):
// tile cp, row n = G row n - 64 cp.  G is 256 rows of 128 bytes (SW128).
constexpr int kGRows = 256;
constexpr int kGBytes = kGRows * 128;
// G rows are 16-byte copies out of 8 phase-shifted BF16 copies of the
// step's kernel slice, s_p[m] = s(m + p), m < kRevLen
constexpr int kRevLen = 192;
constexpr size_t kOffA = 0;
constexpr size_t kOffB = kOffA + (size_t)kStages * kStageBytes;
constexpr size_t kOffO = kOffB + (size_t)2 * kGBytes;
constexpr size_t kOffRev = kOffO + (size_t)4 * 2 * gemm::kOutTileBytes;
constexpr size_t kOffBar = kOffRev + (size_t)2 * 8 * kRevLen * 2;
constexpr size_t kSmem = 1024 + kOffBar + 256;
static_assert(kSmem <= 227 * 1024, "shared memory");

// chunks per (row, frame tile): 2 per column tile, one for the right halo and
// one zero chunk so that every stage is a whole chunk pair
__host__ __device__ inline int n_chunks(int nx) {
    return 2 * ((nx + gemm::kN - 1) / gemm::kN) + 2;
}
}  // namespace gemm2

size_t band_pack_bytes(int nz, int nx, int nf) {
    return (size_t)nz * ((nf + gemm::kM - 1) / gemm::kM) * gemm2::n_chunks(nx) * gemm::kChunkBytes;
}

// in [nf][nz][nx] BF16 -> packed [nz][nm][nq] chunk images.  One block per
// chunk image (row z, frame tile m, chunk q); each thread moves 16-byte pieces
// (8 columns of one frame), 8 consecutive threads one 128-byte frame row.
__global__ void __launch_bounds__(256) tidas_band_pack_kernel(const __nv_bfloat16* __restrict__ in,
                                                              uint8_t* __restrict__ packed, int nz,
                                                              int nx, int nf, int nm, int nq) {
    const int q = blockIdx.x % nq;
    const int zm = blockIdx.x / nq;  // z * nm + m
    const int m = zm % nm, z = zm / nm;
    uint8_t* const dst = packed + (size_t)blockIdx.x * gemm::kChunkBytes;
    for (int u = threadIdx.x; u < gemm::kM * 8; u += blockDim.x) {
        const int j = u & 7, f = u >> 3;
        const int x0 = gemm::kKC * q - 32 + 8 * j;
        const int fr = m * gemm::kM + f;
        uint4 v = make_uint4(0, 0, 0, 0);
        if (fr < nf && x0 >= 0 && x0 < nx)
            v = __ldg(reinterpret_cast<const uint4*>(in + ((size_t)fr * nz + z) * nx + x0));
        *reinterpret_cast<uint4*>(dst + sw128_offset(f, 8 * j)) = v;
    }
}

__device__ __forceinline__ void u_range2d(int z, int kz, int nz, bool adjoint, int& lo, int& hi) {
    const int cz = kz / 2;
    if (adjoint) {
        lo = max(0, cz - z);
        hi = min(kz - 1, nz - 1 - z + cz);
    } else {
        lo = max(0, z + cz - (nz - 1));
        hi = min(kz - 1, z + cz);
    }
}

__global__ void __launch_bounds__(gemm2::kThreads, 1)
    tidas_gemm2d_kernel(const uint8_t* __restrict__ packed,
                        const __grid_constant__ CUtensorMap tmap_out, const float* __restrict__ kern,
                        int kz, int taps, int adjoint, int nz, int nx, int nf) {
    using namespace gemm;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = smem_align1024(smem_raw);
    uint8_t* sA = base + gemm2::kOffA;  // [stage] BF16 input chunks
    uint8_t* sB = base + gemm2::kOffB;  // [buf] band matrix G
    uint8_t* sO = base + gemm2::kOffO;  // [epilogue warp][2] output staging tiles
    __nv_bfloat16* s_rev = (__nv_bfloat16*)(base + gemm2::kOffRev);  // [buf][8][kRevLen]
    uint64_t* full = (uint64_t*)(base + gemm2::kOffBar);
    uint64_t* empty = full + gemm2::kStages;
    uint64_t* b_full = empty + gemm2::kStages;
    uint64_t* b_empty = b_full + 2;
    uint64_t* acc_full = b_empty + 2;
    uint64_t* acc_empty = acc_full + 2;
    uint32_t* tmem_slot = (uint32_t*)(acc_empty + 2);
    volatile int* s_abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cz = kz / 2;
    const int ntiles = (nx + kN - 1) / kN;
    const int nh = (ntiles + kTilesPerItem - 1) / kTilesPerItem;
    const int nm = (nf + kM - 1) / kM;
    const int nq = gemm2::n_chunks(nx);
    const int total = nz * nm * nh;
    // items strided over the grid: the CTAs work on neighbouring rows at the
    // same time, so that each input row is fetched from DRAM about once and
    // its kz uses hit L2
    const int it_begin = blockIdx.x, it_step = gridDim.x;

    if (threadIdx.x == 0) {
        // the two MMA issuers both release stages, bands and accumulators
        for (int s = 0; s < gemm2::kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 2);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&b_full[s], gemm2::kBuilders);
            mbar_init(&b_empty[s], 2);
            mbar_init(&acc_full[s], 2);
            mbar_init(&acc_empty[s], 4);
        }
        *s_abort = 0;
        fence_barrier_init();
        prefetch_tensormap(&tmap_out);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ bulk-copy producer
        if (lane == 0) {
            uint32_t st = 0, ph = 0;
            int issued = 0;
            bool stop = false;
            for (int it = it_begin; it < total && !stop; it += it_step) {
                const Item I = decode(it, nh, nm, ntiles);
                int lo, hi;
                u_range2d(I.z, kz, nz, adjoint, lo, hi);
                for (int u = lo; u <= hi && !stop; ++u) {
                    const int j = adjoint ? I.z + u - cz : I.z - u + cz;
                    const uint8_t* src =
                        packed + ((size_t)j * nm + I.m0 / kM) * nq * (size_t)kChunkBytes;
                    // chunk pairs (2 s0 + 2 p, + 1), p = 0 .. s1 - s0
                    for (int c = 2 * I.s0; c <= 2 * I.s1; c += 2) {
                        if (!mbar_wait_or_abort(&empty[st], ph ^ 1, s_abort, &g_wait_error,
                                                kWaitEmpty)) {
                            stop = true;
                            break;
                        }
                        mbar_arrive_expect_tx(&full[st], gemm2::kStageBytes);
                        bulk_load(sA + st * gemm2::kStageBytes, src + (size_t)c * kChunkBytes,
                                  gemm2::kStageBytes, &full[st]);
                        if (++st == (uint32_t)gemm2::kStages) { st = 0; ph ^= 1; }
                        ++issued;
                    }
                }
            }
            if (*s_abort) {
                // let issued copies land before shared memory is released
                for (int q = 0; q < min(issued, gemm2::kStages); ++q) {
                    st = (st == 0) ? gemm2::kStages - 1 : st - 1;
                    if (st == (uint32_t)gemm2::kStages - 1) ph ^= 1;
                    mbar_wait(&full[st], ph, &g_wait_error, kWaitDrain);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1 || warp == gemm2::kMma2Warp) {
        // ------------------------------------------------- MMA issuers
        // Warp 1 issues the MMAs of the item's first column tile, the other
        // issuer those of the second.  The tensor pipe queues about one MMA,
        // so while one issuer waits on a barrier or commits, the other keeps
        // the pipe fed.  Both wait for every stage and band and release
        // every one, so a stage is refilled only after both are done with it.
        if (lane == 0) {
            const int mine = warp == 1 ? 0 : 1;
            uint32_t st = 0, ph = 0;
            int step = 0, k = 0;
            bool stop = false;
            for (int it = it_begin; it < total && !stop; it += it_step, ++k) {
                const Item I = decode(it, nh, nm, ntiles);
                int lo, hi;
                u_range2d(I.z, kz, nz, adjoint, lo, hi);
                const int ab = k & 1;
                if (!mbar_wait_or_abort(&acc_empty[ab], ((k >> 1) & 1) ^ 1, s_abort, &g_wait_error,
                                        kWaitAccFree))
                    break;
                tc_fence_after();
                for (int u = lo; u <= hi && !stop; ++u, ++step) {
                    const int b = step & 1;
                    if (!mbar_wait_or_abort(&b_full[b], (step >> 1) & 1, s_abort, &g_wait_error,
                                            kWaitB)) {
                        stop = true;
                        break;
                    }
                    tc_fence_after();
                    const uint64_t dg = desc_sw128_kmajor(smem_u32(sB + (size_t)b * gemm2::kGBytes));
                    for (int c2 = 2 * I.s0; c2 <= 2 * I.s1; c2 += 2) {
                        // the bulk copy's completion on full[st] makes the
                        // pair visible to the MMAs; no tcgen05 fence needed
                        if (!mbar_wait_or_abort(&full[st], ph, s_abort, &g_wait_error, kWaitFull)) {
                            stop = true;
                            break;
                        }
                        // descriptors of the pair's two chunks and of the
                        // three windows of G; a K-step adds 32 bytes (2)
                        const uint64_t da = desc_sw128_kmajor(smem_u32(sA + st * gemm2::kStageBytes));
                        const uint32_t acc_u = (u > lo) ? 1u : 0u;
                        // tile tl (relative to s0) from window cp of chunk h
                        auto tile = [&](int tl, int cp, int h) {
                            const uint32_t d = tmem_base + (uint32_t)(ab * kAccCols) + (uint32_t)(tl * kN);
                            const uint64_t a = da + (uint64_t)(h * (kChunkBytes >> 4));
                            const uint64_t bb = dg + (uint64_t)((2 - cp) * (64 * 128 >> 4));
#pragma unroll
                            for (int kk = 0; kk < kKC / 16; ++kk)
                                mma_f16(d, a + 2 * kk, bb + 2 * kk, kIdesc,
                                        (kk > 0 || cp > 0) ? 1u : acc_u);
                        };
                        // the pair is chunks 2 (s0 + t0), + 1; tile `mine` takes
                        // windows 0 and 1 of pair t0 = mine and window 2 of the next
                        const int t0 = c2 / 2 - I.s0;
                        if (mine < I.s1 - I.s0) {
                            if (t0 == mine) {
                                tile(mine, 0, 0);
                                tile(mine, 1, 1);
                            } else if (t0 == mine + 1) {
                                tile(mine, 2, 0);
                            }
                        }
                        mma_commit(&empty[st]);
                        if (++st == (uint32_t)gemm2::kStages) { st = 0; ph ^= 1; }
                    }
                    mma_commit(&b_empty[b]);
                }
                if (stop) break;
                mma_commit(&acc_full[ab]);
            }
        }
        __syncwarp();
    } else if (warp < 6) {
        // ------------------------------------------------------ epilogue
        const int quarter = warp & 3;  // tensor-memory lanes 32*quarter .. +31
        uint8_t* stage_buf = sO + (size_t)(warp - 2) * 2 * kOutTileBytes;
        int k = 0, q = 0;
        for (int it = it_begin; it < total; it += it_step, ++k) {
            const Item I = decode(it, nh, nm, ntiles);
            const int ab = k & 1;
            if (!mbar_wait_or_abort(&acc_full[ab], (k >> 1) & 1, s_abort, &g_wait_error, kWaitAcc))
                break;
            tc_fence_after();
            for (int s = I.s0; s < I.s1; ++s) {
#pragma unroll 1
                for (int j = 0; j < kN / 32; ++j, ++q) {
                    uint32_t r[32];
                    tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                           (uint32_t)(ab * kAccCols + (s - I.s0) * kN + j * 32),
                                       r);
                    tmem_ld_wait();
                    uint8_t* tile = stage_buf + (q & 1) * kOutTileBytes;
                    if (lane == 0) bulk_wait_read<1>();
                    __syncwarp();
#pragma unroll
                    for (int c4 = 0; c4 < 8; ++c4)
                        *reinterpret_cast<uint4*>(tile + lane * 128 + ((c4 ^ (lane & 7)) << 4)) =
                            make_uint4(r[4 * c4], r[4 * c4 + 1], r[4 * c4 + 2], r[4 * c4 + 3]);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_3d(&tmap_out, tile, s * kN + j * 32, I.z, I.m0 + quarter * 32);
                        bulk_commit();
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ab]);
        }
        if (lane == 0) bulk_wait<0>();
        __syncwarp();
    } else {
        // ------------------------------- band matrix G of each (item, u)
        // G[r][k] = s(62 - r + k) with s(m) = h[94 + c - m] (forward, value
        // h[r - k + 32 + c]) or h[m - 94 + c] (adjoint, h[k - r - 32 + c]),
        // c = taps / 2.  Rows outside [r_lo, r_hi] are zero for every slice,
        // and so are the phase-copy entries of s outside the taps: both are
        // cleared once, and a step rewrites only the taps and the band rows.
        const int bt = threadIdx.x - 6 * 32;  // 0 .. 32 * kBuilders - 1
        constexpr int kB = 32 * gemm2::kBuilders;
        const int center = taps / 2;
        const int r_lo = adjoint ? center - 31 - taps : -32 - center;
        const int r_hi = adjoint ? 31 + center : 30 - center + taps;
        const int n_rows = r_hi - r_lo + 1;
        for (int idx = bt; idx < 2 * gemm2::kGRows * 8; idx += kB) {
            const int b = idx / (gemm2::kGRows * 8), row = (idx / 8) % gemm2::kGRows;
            const int r = row - 128;
            if (r < r_lo || r > r_hi)
                *reinterpret_cast<uint4*>(sB + (size_t)b * gemm2::kGBytes + row * 128 +
                                          (idx % 8) * 16) = make_uint4(0, 0, 0, 0);
        }
        for (int idx = bt; idx < 2 * 8 * gemm2::kRevLen / 2; idx += kB)
            reinterpret_cast<uint32_t*>(s_rev)[idx] = 0u;
        // tap bt of a slice sits at s index m_t, i.e. at m_t - p in copy p
        const int m_t = adjoint ? bt + 94 - center : 94 + center - bt;
        named_bar_sync<1>(kB);
        // the slice value this thread carries into the next step
        auto slice_tap = [&](int it, int u) -> float {
            if (bt >= taps || it >= total) return 0.f;
            const int z = it / (nh * nm);
            const int krow = adjoint ? z : z - u + cz;
            return __ldg(kern + ((size_t)krow * kz + u) * taps + bt);
        };
        int it = it_begin, lo = 0, hi = -1, u = 0;
        if (it < total) {
            u_range2d(decode(it, nh, nm, ntiles).z, kz, nz, adjoint, lo, hi);
            u = lo;
        }
        float tap = slice_tap(it, u);
        for (int step = 0; it < total; ++step) {
            const int b = step & 1;
            const bool ok = mbar_wait_or_abort(&b_empty[b], ((step >> 1) & 1) ^ 1, s_abort,
                                               &g_wait_error, kWaitB);
            __nv_bfloat16* rev = s_rev + b * 8 * gemm2::kRevLen;
            if (ok && bt < taps) {
                const __nv_bfloat16 hv = __float2bfloat16_rn(tap);
#pragma unroll
                for (int p = 0; p < 8; ++p) rev[p * gemm2::kRevLen + m_t - p] = hv;
            }
            // the taps are in; leave together if any builder or role gave up
            if (named_bar_or<1>(kB, !ok || *s_abort)) break;
            // next step's slice, loaded while this one is built
            if (u < hi) {
                ++u;
            } else {
                it += it_step;
                if (it < total) {
                    u_range2d(decode(it, nh, nm, ntiles).z, kz, nz, adjoint, lo, hi);
                    u = lo;
                }
            }
            tap = slice_tap(it, u);
            uint8_t* dst = sB + (size_t)b * gemm2::kGBytes;
            for (int idx = bt; idx < n_rows * 8; idx += kB) {
                const int r = r_lo + idx / 8, j = idx % 8;
                const int m0 = 62 - r + 8 * j;  // 0 .. 181
                const uint4 v = *reinterpret_cast<const uint4*>(
                    rev + (m0 & 7) * gemm2::kRevLen + (m0 & ~7));
                const int row = r + 128;
                *reinterpret_cast<uint4*>(dst + row * 128 + ((j ^ (row & 7)) << 4)) = v;
            }
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&b_full[b]);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, kTmemCols);
    }
}

int launch_tidas_gemm2d(const float* kern, int kz, int taps, bool adjoint, int nz, int nx,
                        const void* in, float* out, int nf, void* workspace, size_t ws_bytes,
                        cudaStream_t st) {
    CUtensorMap map_out;
    int rc = make_map_3d(&map_out, out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nz, nx, nf, 32, 32,
                         CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    const size_t need = band_pack_bytes(nz, nx, nf);
    uint8_t* packed = (uint8_t*)workspace;
    if (packed) {
        if (ws_bytes < need)
            return set_error(TIDAS_ERR_ARG, "tidas 2D GEMM: workspace of %zu bytes, need %zu",
                             ws_bytes, need);
        if ((uintptr_t)packed % 16)
            return set_error(TIDAS_ERR_ARG, "tidas 2D GEMM: workspace must be 16-byte aligned");
    } else {
        TIDAS_CUDA(cudaMallocAsync((void**)&packed, need, st));
    }
    const int nm = (nf + gemm::kM - 1) / gemm::kM, nq = gemm2::n_chunks(nx);
    const size_t images = (size_t)nz * nm * nq;
    if (images > (size_t)INT_MAX) {
        rc = set_error(TIDAS_ERR_UNSUPPORTED, "tidas 2D GEMM: %zu chunk images", images);
    } else {
        tidas_band_pack_kernel<<<(unsigned)images, 256, 0, st>>>((const __nv_bfloat16*)in, packed,
                                                                 nz, nx, nf, nm, nq);
        rc = check_launch("tidas_band_pack_kernel");
    }
    if (rc == TIDAS_OK) {
        const int ntiles = (nx + gemm::kN - 1) / gemm::kN;
        const int items = nz * nm * ((ntiles + gemm::kTilesPerItem - 1) / gemm::kTilesPerItem);
        const int grid = items < sm_count() ? items : sm_count();
        rc = check_cuda(cudaFuncSetAttribute(tidas_gemm2d_kernel,
                                             cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)gemm2::kSmem),
                        "cudaFuncSetAttribute(tidas_gemm2d_kernel)");
        if (rc == TIDAS_OK) {
            tidas_gemm2d_kernel<<<grid, gemm2::kThreads, gemm2::kSmem, st>>>(
                packed, map_out, kern, kz, taps, adjoint ? 1 : 0, nz, nx, nf);
            rc = check_launch("tidas_gemm2d_kernel");
        }
    }
    if (!workspace) cudaFreeAsync(packed, st);
    return rc;
}

// ------------------------------------ spatially varying band kernels (tcgen05)
// Eq. (2.13) with a kernel per pixel (each input pixel adds its own
// single-scatterer image):
//   y[f][i][x] = sum_{u,t} K[j][s][u][t] r[f][j][s],  j = i - u + kz/2,  s = x - t + taps/2.
// Work item = (output row i, 128-column tile, up to two 128-frame tiles).
// The K loop runs over the band slices u and the tile's input chunks
// q = 2 xt + c, c = 0..2, whose columns [64 q - 32, 64 q + 32) cover every s
// the tile reads.  A step multiplies the packed input chunk of row j (the 2D
// band GEMM's operand image, 128 frames x 64 columns per frame tile) by a B
// tile that the builder warps write from the kernels of the chunk's pixels,
//     B[x][s] = K[j][s][u][x - s + taps/2]   (zero outside the taps),
// 128 output columns x 64 input columns, K-major, 128-byte swizzle: row x of
// B collects, for each input pixel, the tap that reaches x.  The kernel
// varies from pixel to pixel, so unlike the shift-invariant kernels no B
// tile serves two steps.  The chunk's kernel slice (64 pixels x slice u,
// FP32) arrives in the step's stage by one TMA box beside the input chunks,
// so that the builders read shared memory (consecutive lanes take
// consecutive output columns, i.e. consecutive taps of one pixel: distinct
// banks) and never wait on DRAM.
//   warp 0      producer: input chunks (bulk copies) and kernel slices (TMA)
//               into a 3-stage ring
//   warp 1      tensor-memory owner; lane 0 issues the MMAs
//   warps 2-9   B tiles (double buffered)
//   warps 10-13 epilogue: tensor memory -> swizzled staging tile -> TMA store
// Accumulators (two frame tiles x 128 columns) are double buffered, so the
// epilogue of one item overlaps the MMAs of the next.
namespace vgem {
constexpr int kStages = 3;
constexpr int kMaxFT = 2;
constexpr int kKOff = kMaxFT * gemm::kChunkBytes;         // kernel slice within a stage
constexpr int kKBytes = 64 * 64 * 4;                      // 64 pixels x <= 64 FP32 (or BF16) taps
constexpr int kStageBytes = kKOff + kKBytes;              // 48 KB
constexpr int kBBufs = 2;
constexpr int kBuilders = 8;
constexpr int kBuilder0 = 2;
constexpr int kEpi0 = kBuilder0 + kBuilders;  // 10
constexpr int kWarps = kEpi0 + 4;
constexpr int kThreads = 32 * kWarps;
constexpr uint32_t kAccCols = kMaxFT * gemm::kN;  // 256
constexpr uint32_t kTmemCols = 2 * kAccCols;      // 512
constexpr size_t kOffA = 0;
constexpr size_t kOffB = kOffA + (size_t)kStages * kStageBytes;
constexpr size_t kOffO = kOffB + (size_t)kBBufs * gemm::kBTileBytes;
constexpr size_t kOffBar = kOffO + (size_t)4 * 2 * gemm::kOutTileBytes;
constexpr size_t kSmem = 1024 + kOffBar + 256;
static_assert(kSmem <= 227 * 1024, "shared memory");
constexpr int kWaitEmpty = 111, kWaitFull = 112, kWaitB = 113, kWaitBFree = 114, kWaitAcc = 115,
              kWaitAccFree = 116, kWaitDrain = 117, kWaitDone = 118;

struct VItem {
    int i, xt, ft0, nft, lo, hi, nc;
};
// items: row fastest, so that neighbouring CTAs share input rows in L2
__device__ __forceinline__ VItem vdecode(int it, int nz, int ntiles, int nm, int kz, int nx) {
    VItem v;
    v.i = it % nz;
    v.xt = (it / nz) % ntiles;
    v.ft0 = (it / (nz * ntiles)) * kMaxFT;
    v.nft = min(kMaxFT, nm - v.ft0);
    u_range2d(v.i, kz, nz, false, v.lo, v.hi);
    // input chunks of the tile that start inside the row
    v.nc = 0;
    for (int c = 0; c < 3; ++c)
        if (64 * (2 * v.xt + c) - 32 < nx) v.nc = c + 1;
    return v;
}
}  // namespace vgem

// K16: the per-pixel kernels are BF16 (half of each stage's kernel slot is
// used); otherwise FP32, rounded to BF16 by the builders.
template <bool K16>
__global__ void __launch_bounds__(vgem::kThreads, 1)
    tidas_varying_gemm_kernel(const uint8_t* __restrict__ packed,
                              const __grid_constant__ CUtensorMap tmap_out,
                              const __grid_constant__ CUtensorMap tmap_k, int boxw, int kz,
                              int taps, int nz, int nx, int nf) {
    using namespace gemm;
    using namespace vgem;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = smem_align1024(smem_raw);
    uint8_t* sA = base + vgem::kOffA;
    uint8_t* sB = base + vgem::kOffB;
    uint8_t* sO = base + vgem::kOffO;
    uint64_t* full = (uint64_t*)(base + vgem::kOffBar);
    uint64_t* empty = full + vgem::kStages;
    uint64_t* b_full = empty + vgem::kStages;
    uint64_t* b_empty = b_full + kBBufs;
    uint64_t* acc_full = b_empty + kBBufs;
    uint64_t* acc_empty = acc_full + 2;
    uint64_t* done = acc_empty + 2;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* s_abort = (volatile int*)(tmem_slot + 1);

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int cz = kz / 2, cx = taps / 2;
    const int ntiles = (nx + kN - 1) / kN;
    const int nm = (nf + kM - 1) / kM;
    const int nq = gemm2::n_chunks(nx);
    const int total = nz * ntiles * ((nm + kMaxFT - 1) / kMaxFT);
    const int it_begin = blockIdx.x, it_step = gridDim.x;

    if (threadIdx.x == 0) {
        for (int s = 0; s < vgem::kStages; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int s = 0; s < kBBufs; ++s) {
            mbar_init(&b_full[s], kBuilders);
            mbar_init(&b_empty[s], 1);
        }
        for (int s = 0; s < 2; ++s) {
            mbar_init(&acc_full[s], 1);
            mbar_init(&acc_empty[s], 4);
        }
        mbar_init(done, 1);
        *s_abort = 0;
        fence_barrier_init();
        prefetch_tensormap(&tmap_out);
        prefetch_tensormap(&tmap_k);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, vgem::kTmemCols);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem_base = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------------ bulk-copy producer
        if (lane == 0) {
            uint32_t st = 0, ph = 0;
            int issued = 0;
            bool stop = false;
            for (int it = it_begin; it < total && !stop; it += it_step) {
                const VItem I = vdecode(it, nz, ntiles, nm, kz, nx);
                for (int u = I.lo; u <= I.hi && !stop; ++u) {
                    const int j = I.i - u + cz;
                    for (int c = 0; c < I.nc; ++c) {
                        if (!mbar_wait_or_abort(&empty[st], ph ^ 1, s_abort, &g_wait_error,
                                                vgem::kWaitEmpty)) {
                            stop = true;
                            break;
                        }
                        mbar_arrive_expect_tx(&full[st],
                                              (uint32_t)(I.nft * kChunkBytes + boxw * 64 * (K16 ? 2 : 4)));
                        const int q = 2 * I.xt + c;
                        for (int f = 0; f < I.nft; ++f)
                            bulk_load(sA + st * vgem::kStageBytes + f * kChunkBytes,
                                      packed + (((size_t)j * nm + I.ft0 + f) * nq + q) * kChunkBytes,
                                      kChunkBytes, &full[st]);
                        // slice u of the chunk's 64 pixels j nx + 64 q - 32 ..; pixels
                        // past either end of the grid are zero-filled, those of a
                        // neighbouring row are masked by the builders
                        tma_load_3d(sA + st * vgem::kStageBytes + vgem::kKOff, &tmap_k, &full[st],
                                    0, u, j * nx + 64 * q - 32);
                        if (++st == (uint32_t)vgem::kStages) { st = 0; ph ^= 1; }
                        ++issued;
                    }
                }
            }
            if (*s_abort) {
                // let issued copies land before shared memory is released
                for (int k = 0; k < min(issued, vgem::kStages); ++k) {
                    st = (st == 0) ? vgem::kStages - 1 : st - 1;
                    if (st == (uint32_t)vgem::kStages - 1) ph ^= 1;
                    mbar_wait(&full[st], ph, &g_wait_error, vgem::kWaitDrain);
                }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------ MMA issuer
        if (lane == 0) {
            uint32_t st = 0, ph = 0;
            int step = 0, k = 0;
            bool stop = false;
            for (int it = it_begin; it < total && !stop; it += it_step, ++k) {
                const VItem I = vdecode(it, nz, ntiles, nm, kz, nx);
                const int ab = k & 1;
                if (!mbar_wait_or_abort(&acc_empty[ab], ((k >> 1) & 1) ^ 1, s_abort, &g_wait_error,
                                        vgem::kWaitAccFree))
                    break;
                tc_fence_after();
                bool first = true;
                for (int u = I.lo; u <= I.hi && !stop; ++u) {
                    for (int c = 0; c < I.nc; ++c, ++step) {
                        const int b = step & 1;
                        if (!mbar_wait_or_abort(&full[st], ph, s_abort, &g_wait_error,
                                                vgem::kWaitFull) ||
                            !mbar_wait_or_abort(&b_full[b], (step >> 1) & 1, s_abort,
                                                &g_wait_error, vgem::kWaitB)) {
                            stop = true;
                            break;
                        }
                        tc_fence_after();
                        const uint64_t db = desc_sw128_kmajor(smem_u32(sB + b * kBTileBytes));
                        for (int f = 0; f < I.nft; ++f) {
                            const uint64_t da = desc_sw128_kmajor(
                                smem_u32(sA + st * vgem::kStageBytes + f * kChunkBytes));
                            const uint32_t d = tmem_base + (uint32_t)(ab * vgem::kAccCols) +
                                               (uint32_t)(f * kN);
#pragma unroll
                            for (int kk = 0; kk < kKC / 16; ++kk)
                                mma_f16(d, da + 2 * kk, db + 2 * kk, kIdesc,
                                        (first && kk == 0) ? 0u : 1u);
                        }
                        first = false;
                        mma_commit(&empty[st]);
                        mma_commit(&b_empty[b]);
                        if (++st == (uint32_t)vgem::kStages) { st = 0; ph ^= 1; }
                    }
                }
                if (stop) break;
                mma_commit(&acc_full[ab]);
            }
            // every MMA this thread issued has completed before tensor memory
            // is released (also after an abort)
            mma_commit(done);
            mbar_wait(done, 0, &g_wait_error, vgem::kWaitDone);
        }
        __syncwarp();
    } else if (warp < kEpi0) {
        // --------------------------------------------------------- B tiles
        // thread: output row x = 32 (wb % 4) + lane of the tile, 16-byte
        // chunks 4 (wb / 4) .. + 3 (input columns 8 k16 .. + 7 of the chunk)
        const int wb = warp - kBuilder0;
        const int x_rel = 32 * (wb & 3) + lane;
        const int k16_0 = 4 * (wb >> 2);
        int step = 0;
        uint32_t st = 0, ph = 0;
        bool stop = false;
        for (int it = it_begin; it < total && !stop; it += it_step) {
            const VItem I = vdecode(it, nz, ntiles, nm, kz, nx);
            const int x = kN * I.xt + x_rel;
            for (int u = I.lo; u <= I.hi && !stop; ++u) {
                for (int c = 0; c < I.nc; ++c, ++step) {
                    const int b = step & 1;
                    const int s0 = 64 * (2 * I.xt + c) - 32;
                    // the step's kernel slice has landed in its stage, and the
                    // B buffer of two steps ago has been read by its MMAs
                    bool ok = mbar_wait_or_abort(&full[st], ph, s_abort, &g_wait_error,
                                                 vgem::kWaitFull) &&
                              mbar_wait_or_abort(&b_empty[b], ((step >> 1) & 1) ^ 1, s_abort,
                                                 &g_wait_error, vgem::kWaitBFree);
                    if (ok) {
                        const uint8_t* kslot = sA + st * vgem::kStageBytes + vgem::kKOff;
                        // the 32 BF16 weights of this thread's four 16-byte chunks,
                        // as pairs: word e holds inputs 2 e, 2 e + 1
                        uint32_t wd[16];
                        if (K16) {
                            const uint16_t* ks = reinterpret_cast<const uint16_t*>(kslot);
#pragma unroll
                            for (int e = 0; e < 16; ++e) {
                                uint32_t pr[2];
#pragma unroll
                                for (int k = 0; k < 2; ++k) {
                                    const int sl = 8 * k16_0 + 2 * e + k;  // pixel s0 + sl of the slice
                                    const int sx = s0 + sl;
                                    const int t = x - sx + cx;
                                    pr[k] = (t >= 0 && t < taps && sx >= 0 && sx < nx)
                                                ? (uint32_t)ks[sl * boxw + t] : 0u;
                                }
                                wd[e] = pr[0] | (pr[1] << 16);
                            }
                        } else {
                            const float* ks = reinterpret_cast<const float*>(kslot);
                            float v[32];
#pragma unroll
                            for (int e = 0; e < 32; ++e) {
                                const int sl = 8 * k16_0 + e;  // pixel s0 + sl of the slice
                                const int sx = s0 + sl;
                                const int t = x - sx + cx;
                                v[e] = (t >= 0 && t < taps && sx >= 0 && sx < nx) ? ks[sl * boxw + t]
                                                                                  : 0.f;
                            }
#pragma unroll
                            for (int e = 0; e < 16; ++e) {
                                const __nv_bfloat162 p2 = __floats2bfloat162_rn(v[2 * e], v[2 * e + 1]);
                                wd[e] = *reinterpret_cast<const uint32_t*>(&p2);
                            }
                        }
                        uint8_t* dst = sB + b * kBTileBytes;
#pragma unroll
                        for (int h = 0; h < 4; ++h)
                            *reinterpret_cast<uint4*>(dst + sw128_offset(x_rel, 8 * (k16_0 + h))) =
                                make_uint4(wd[4 * h], wd[4 * h + 1], wd[4 * h + 2], wd[4 * h + 3]);
                        fence_proxy_async_smem();
                    }
                    __syncwarp();
                    if (__any_sync(0xffffffffu, !ok)) {
                        stop = true;
                        break;
                    }
                    if (lane == 0) mbar_arrive(&b_full[b]);
                    if (++st == (uint32_t)vgem::kStages) { st = 0; ph ^= 1; }
                }
            }
        }
    } else {
        // ------------------------------------------------------- epilogue
        const int quarter = warp & 3;  // tensor-memory lanes 32 quarter .. + 31
        uint8_t* stage_buf = sO + (size_t)(warp - kEpi0) * 2 * kOutTileBytes;
        int k = 0, q = 0;
        for (int it = it_begin; it < total; it += it_step, ++k) {
            const VItem I = vdecode(it, nz, ntiles, nm, kz, nx);
            const int ab = k & 1;
            if (!mbar_wait_or_abort(&acc_full[ab], (k >> 1) & 1, s_abort, &g_wait_error,
                                    vgem::kWaitAcc))
                break;
            tc_fence_after();
            for (int f = 0; f < I.nft; ++f) {
#pragma unroll 1
                for (int jc = 0; jc < kN / 32; ++jc, ++q) {
                    uint32_t r[32];
                    tmem_ld_32x32b_x32(tmem_base + ((uint32_t)(quarter * 32) << 16) +
                                           (uint32_t)(ab * vgem::kAccCols + f * kN + jc * 32),
                                       r);
                    tmem_ld_wait();
                    uint8_t* tile = stage_buf + (q & 1) * kOutTileBytes;
                    if (lane == 0) bulk_wait_read<1>();
                    __syncwarp();
#pragma unroll
                    for (int c4 = 0; c4 < 8; ++c4)
                        *reinterpret_cast<uint4*>(tile + lane * 128 + ((c4 ^ (lane & 7)) << 4)) =
                            make_uint4(r[4 * c4], r[4 * c4 + 1], r[4 * c4 + 2], r[4 * c4 + 3]);
                    fence_proxy_async_smem();
                    __syncwarp();
                    if (lane == 0) {
                        tma_store_3d(&tmap_out, tile, kN * I.xt + jc * 32, I.i,
                                     (I.ft0 + f) * kM + quarter * 32);
                        bulk_commit();
                    }
                }
            }
            tc_fence_before();
            __syncwarp();
            if (lane == 0) mbar_arrive(&acc_empty[ab]);
        }
        if (lane == 0) bulk_wait<0>();
        __syncwarp();
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem_base, vgem::kTmemCols);
    }
}

// rows [rows][ld] -> [rows][ldp] (the first taps columns, zero padding);
// T is float or a 16-bit storage type
template <typename T>
__global__ void pad_rows_kernel(const T* __restrict__ in, int ld, int taps, long long rows,
                                T* __restrict__ out, int ldp) {
    const long long n = rows * ldp;
    for (long long q = (long long)blockIdx.x * blockDim.x + threadIdx.x; q < n;
         q += (long long)gridDim.x * blockDim.x) {
        const long long r = q / ldp;
        const int t = (int)(q - r * ldp);
        out[q] = t < taps ? in[r * ld + t] : T(0);
    }
}

// kern: FP32 (k16 false) or BF16 (k16 true) per-pixel kernels [nz][nx][kz][ld]
int launch_tidas_varying_gemm(const void* kern, bool k16, int ld, int kz, int taps, int nz, int nx,
                              const void* in, float* out, int nf, cudaStream_t st) {
    CUtensorMap map_out, map_k;
    int rc = make_map_3d(&map_out, out, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 4, nz, nx, nf, 32, 32,
                         CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    const int nm = (nf + gemm::kM - 1) / gemm::kM, nq = gemm2::n_chunks(nx);
    const size_t images = (size_t)nz * nm * nq;
    if (images > (size_t)INT_MAX)
        return set_error(TIDAS_ERR_UNSUPPORTED, "tidas varying GEMM: %zu chunk images", images);
    // kernel rows of a pitch that TMA cannot address (not a multiple of 16
    // bytes) are first copied to a padded scratch
    const long long krows = (long long)nz * nx * kz;
    const int esz = k16 ? 2 : 4, per16 = 16 / esz;  // elements per 16 bytes
    void* kpad = nullptr;
    int kld = ld;
    if (ld % per16) {
        kld = (taps + per16 - 1) / per16 * per16;
        TIDAS_CUDA(cudaMallocAsync(&kpad, (size_t)esz * krows * kld, st));
        if (k16)
            pad_rows_kernel<uint16_t><<<152 * 8, 256, 0, st>>>((const uint16_t*)kern, ld, taps, krows,
                                                               (uint16_t*)kpad, kld);
        else
            pad_rows_kernel<float><<<152 * 8, 256, 0, st>>>((const float*)kern, ld, taps, krows,
                                                            (float*)kpad, kld);
        rc = check_launch("pad_rows_kernel");
        kern = kpad;
    }
    const int boxw = kld < 64 ? kld : 64;
    if (rc == TIDAS_OK) {
        // the kernels as [pixel][slice][kld]: box = boxw taps x 1 slice x 64 pixels
        EncodeTiledFn enc = encode_fn();
        if (!enc) {
            rc = set_error(TIDAS_ERR_CUDA, "cuTensorMapEncodeTiled unavailable");
        } else {
            cuuint64_t dims[3] = {(cuuint64_t)kld, (cuuint64_t)kz, (cuuint64_t)nz * nx};
            cuuint64_t strides[2] = {(cuuint64_t)kld * esz, (cuuint64_t)kz * kld * esz};
            cuuint32_t box[3] = {(cuuint32_t)boxw, 1u, 64u};
            cuuint32_t estr[3] = {1u, 1u, 1u};
            CUresult r = enc(&map_k, k16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32,
                             3, const_cast<void*>(kern),
                             dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE,
                             CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_128B,
                             CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
            if (r != CUDA_SUCCESS)
                rc = set_error(TIDAS_ERR_CUDA, "cuTensorMapEncodeTiled (kernels) failed (%d)",
                               (int)r);
        }
    }
    uint8_t* packed = nullptr;
    if (rc == TIDAS_OK) {
        cudaError_t e = cudaMallocAsync((void**)&packed, band_pack_bytes(nz, nx, nf), st);
        if (e != cudaSuccess) {
            rc = check_cuda(e, "cudaMallocAsync(varying GEMM operands)");
            packed = nullptr;
        }
    }
    if (rc == TIDAS_OK) {
        tidas_band_pack_kernel<<<(unsigned)images, 256, 0, st>>>((const __nv_bfloat16*)in, packed,
                                                                 nz, nx, nf, nm, nq);
        rc = check_launch("tidas_band_pack_kernel");
    }
    if (rc == TIDAS_OK) {
        const int ntiles = (nx + gemm::kN - 1) / gemm::kN;
        const int items = nz * ntiles * ((nm + vgem::kMaxFT - 1) / vgem::kMaxFT);
        const int grid = items < sm_count() ? items : sm_count();
        auto kfn = k16 ? tidas_varying_gemm_kernel<true> : tidas_varying_gemm_kernel<false>;
        rc = check_cuda(cudaFuncSetAttribute(kfn, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             (int)vgem::kSmem),
                        "cudaFuncSetAttribute(tidas_varying_gemm_kernel)");
        if (rc == TIDAS_OK) {
            kfn<<<grid, vgem::kThreads, vgem::kSmem, st>>>(packed, map_out, map_k, boxw, kz, taps,
                                                           nz, nx, nf);
            rc = check_launch("tidas_varying_gemm_kernel");
        }
    }
    if (packed) cudaFreeAsync(packed, st);
    if (kpad) cudaFreeAsync(kpad, st);
    return rc;
}

}  // namespace tidas

namespace tidas {
int read_clear_mlp_wait_flag(int* v);
int read_clear_das_tc_wait_flag(int* v);
int read_clear_mlp_infer_wait_flag(int* v);
}

extern "C" int tidas_device_status(int32_t* status) {
    TIDAS_REQUIRE(status, "tidas_device_status: null argument");
    TIDAS_CUDA(cudaDeviceSynchronize());
    int v = 0, zero = 0;
    TIDAS_CUDA(cudaMemcpyFromSymbol(&v, tidas::g_wait_error, sizeof(int)));
    TIDAS_CUDA(cudaMemcpyToSymbol(tidas::g_wait_error, &zero, sizeof(int)));
    int v2 = 0, v3 = 0, v4 = 0;
    int rc = tidas::read_clear_mlp_wait_flag(&v2);
    if (rc) return rc;
    rc = tidas::read_clear_das_tc_wait_flag(&v3);
    if (rc) return rc;
    rc = tidas::read_clear_mlp_infer_wait_flag(&v4);
    if (rc) return rc;
    if (v == 0) v = v2;
    if (v == 0) v = v3;
    if (v == 0) v = v4;
    *status = v;
    if (v != 0)
        return tidas::set_error(TIDAS_ERR_TIMEOUT, "a bounded device wait gave up (code %d)", v);
    return TIDAS_OK;
}
