// Delay and Sum (Eq. (2.2)) for batches of FP16 channel data on the tcgen05
// tensor cores.
//
// For a tile of 128 pixels (16 columns x 8 rows) and a tile of NF frames,
//     img[p, f] = sum_{a,n} sum_k W_an[p, k] * rf[f, a, n, k0_an + k],
// where row p of W_an holds the apodized interpolation weights
// w_n(p) * K(u - m) of the (2 or 4) samples m that pixel p reads, placed at
// columns m - k0_an.  Over one tile every (angle, element) pair reads a
// window of fewer than 64 consecutive samples, so each pair is a dense
// 128 x NF x (<= 64) FP16 contraction accumulated in FP32 tensor memory.
// The window start k0_an (a multiple of 8, for TMA alignment) and the
// number of 16-column K-steps are tabulated per (tile, angle, element) when
// the plan is created.
//
// Warp roles: warp 0 streams channel windows [NF frames x 64 samples] by
// TMA (zero fill outside the record) through a deep ring, so that the L2
// latency of the many small windows is covered; warp 1 owns tensor memory
// and issues the MMAs; warps 2-9 build W_an (two groups of four warps on
// alternate pairs), one pixel per thread, writing and later erasing whole swizzled 16-byte chunks (the
// swizzle spreads the 32 rows of a warp over distinct banks), and finally
// drain the accumulators.
#include <climits>
#include <vector>

#include "common.cuh"
#include "sm103_primitives.cuh"

namespace tidas {
using namespace sm103;

// wait flag of this kernel (read through tidas_device_status)
__device__ int g_das_tc_wait_error = 0;

int read_clear_das_tc_wait_flag(int* v) {
    int zero = 0;
    cudaError_t e = cudaMemcpyFromSymbol(v, g_das_tc_wait_error, sizeof(int));
    if (e == cudaSuccess) e = cudaMemcpyToSymbol(g_das_tc_wait_error, &zero, sizeof(int));
    return check_cuda(e, "das tc wait flag");
}

namespace dtc {
constexpr int kTX = 16, kTZ = 8;          // pixel tile
constexpr int kM = kTX * kTZ;             // 128 = UMMA M
constexpr int kKW = 64;                   // window columns (one 128-byte swizzle row)
constexpr int kWStages = 4;               // weight tiles in flight (a power of two)
constexpr int kRStages = 3;               // channel windows in flight
constexpr int kWBytes = kM * kKW * 2;     // 16 KB
// channel stage = NF frames x 128 bytes, sized per launch
__host__ __device__ constexpr int r_bytes(int NF) { return (NF < 32 ? 32 : NF) * kKW * 2; }
__host__ __device__ constexpr size_t smem_bytes(int NF, int A, int NE) {
    return 1024 + (size_t)kWStages * kWBytes + (size_t)kRStages * r_bytes(NF) + 1024 +
           (size_t)kWStages * kM * 4 + (size_t)A * kM * 8 + (size_t)A * NE * 4;
}
}  // namespace dtc

// Place the 4 FP16 weights `v` (packed in 64 bits) at half offset o (0..7)
// of a 32-byte span: lo / hi are the two 16-byte chunks.
__device__ __forceinline__ void place4(uint64_t v, int o, uint4& lo, uint4& hi) {
    const int s = (o & 3) * 16;
    const uint64_t a = v << s, b = s ? v >> (64 - s) : 0ull;
    if (o < 4) {
        lo = make_uint4((uint32_t)a, (uint32_t)(a >> 32), (uint32_t)b, (uint32_t)(b >> 32));
        hi = make_uint4(0, 0, 0, 0);
    } else {
        lo = make_uint4(0, 0, (uint32_t)a, (uint32_t)(a >> 32));
        hi = make_uint4((uint32_t)b, (uint32_t)(b >> 32), 0, 0);
    }
}

// Per-(tile, angle, element) window: entry = k0 * 8 + ksteps (k0 may be
// negative; ksteps 0 means no contributing pixel).  Per tile: element range.
__global__ void das_tc_table_kernel(DasDev d, int tiles_x, int tiles, int* __restrict__ tab,
                                    int2* __restrict__ range, int* __restrict__ bad) {
    const int NE = d.n_elem, A = d.n_angles;
    const long long total = (long long)tiles * A * NE;
    for (long long q = blockIdx.x * (long long)blockDim.x + threadIdx.x; q < total;
         q += (long long)gridDim.x * blockDim.x) {
        const int n = (int)(q % NE);
        const int a = (int)((q / NE) % A);
        const int tile = (int)(q / ((long long)NE * A));
        const int tx = tile % tiles_x, tz = tile / tiles_x;
        int lo = INT_MAX, hi = INT_MIN;
        for (int m = 0; m < dtc::kM; ++m) {
            const int ix = tx * dtc::kTX + (m % dtc::kTX), iz = tz * dtc::kTZ + m / dtc::kTX;
            if (ix >= d.nx || iz >= d.nz) continue;
            const float dxs = __ldg(d.dxs + (size_t)n * d.nx + ix), zs = __ldg(d.zs + iz);
            if (apod_weight(dxs, zs, d.fnum) == 0.f) continue;
            int i;
            float phi;
            pixel_delay(d, a, ix, iz, rx_excess(dxs, zs), i, phi);
            lo = min(lo, i);
            hi = max(hi, i);
        }
        int entry = 0;
        if (lo <= hi) {
            // taps i-1 .. i+2 (cubic) or i .. i+1 (linear), one sample of slack each side
            const int c_lo = lo - 2, c_hi = hi + 3;
            const int k0 = (int)floorf((float)c_lo / 8.f) * 8;
            const int span = c_hi - k0 + 1;
            const int steps = (span + 15) / 16;
            if (steps > 4) atomicExch(bad, 1);
            entry = k0 * 8 + min(steps, 4);
            atomicMin(&range[tile].x, n);
            atomicMax(&range[tile].y, n);
        }
        tab[q] = entry;
    }
}

__global__ void __launch_bounds__(320, 1)
    das_tc_kernel(const __grid_constant__ CUtensorMap tmap, DasDev d, const int* __restrict__ tab,
                  const int2* __restrict__ range, int tiles_x, int nf, int NF,
                  float* __restrict__ img) {
    using namespace dtc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = (uint8_t*)(((uintptr_t)smem_raw + 1023) & ~(uintptr_t)1023);
    const int RB = r_bytes(NF);
    uint8_t* sW = base;
    uint8_t* sR = base + kWStages * kWBytes;
    uint64_t* full_r = (uint64_t*)(sR + kRStages * RB);
    uint64_t* empty_r = full_r + kRStages;
    uint64_t* full_w = empty_r + kRStages;
    uint64_t* empty_w = full_w + kWStages;
    uint64_t* done = empty_w + kWStages;
    uint32_t* tmem_slot = (uint32_t*)(done + 1);
    volatile int* s_abort = (volatile int*)(tmem_slot + 1);
    int* prev = (int*)((uint8_t*)full_r + 1024);              // [kWStages][kM]
    int2* s_base = (int2*)(prev + kWStages * kM);              // [A][kM]: transmit split
    int* s_tab = (int*)(s_base + d.n_angles * kM);             // [pair]: window entries

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int tile = blockIdx.x;
    const int tx = tile % tiles_x, tz = tile / tiles_x;
    const int f0 = blockIdx.y * NF;
    const int A = d.n_angles, NE = d.n_elem;
    const int2 rg = range[tile];
    const int n_lo = rg.x, n_hi = rg.y;
    const int npairs = n_hi >= n_lo ? (n_hi - n_lo + 1) * A : 0;
    const uint32_t tcols = NF <= 32 ? 32 : (NF <= 64 ? 64 : 128);
    const uint32_t idesc = idesc_f16_f32(kM, NF);
    const uint32_t rbytes = (uint32_t)(NF * kKW * 2);

    if (threadIdx.x == 0) {
        for (int s = 0; s < kRStages; ++s) {
            mbar_init(&full_r[s], 1);
            mbar_init(&empty_r[s], 1);
        }
        for (int s = 0; s < kWStages; ++s) {
            mbar_init(&full_w[s], 4);
            mbar_init(&empty_w[s], 1);
        }
        mbar_init(done, 1);
        *s_abort = 0;
        fence_barrier_init();
        prefetch_tensormap(&tmap);
    }
    // zero the weight tiles once; afterwards only written chunks are erased
    for (int i = threadIdx.x; i < kWStages * kWBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sW)[i] = make_uint4(0, 0, 0, 0);
    for (int i = threadIdx.x; i < kWStages * kM; i += blockDim.x) prev[i] = -1;
    // this tile's window entries (pair order: element-major, angle-minor), so
    // that no role waits on a global load per pair
    {
        const int* tt = tab + (size_t)tile * A * NE;
        for (int i = threadIdx.x; i < npairs; i += blockDim.x)
            s_tab[i] = __ldg(tt + (i % A) * NE + n_lo + i / A);
    }
    if (warp == 1) {
        tmem_alloc(tmem_slot, tcols);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        // ------------------------------------------ channel windows by TMA
        if (lane == 0) {
            uint32_t st = 0, ph = 0;
            for (int q = 0; q < npairs && !*s_abort; ++q) {
                const int n = n_lo + q / A, a = q % A;
                const int e = s_tab[q];
                if (!mbar_wait(&empty_r[st], ph ^ 1, &g_das_tc_wait_error, 301)) {
                    *s_abort = 1;
                    break;
                }
                mbar_arrive_expect_tx(&full_r[st], rbytes);
                tma_load_3d(sR + st * RB, &tmap, &full_r[st], e >> 3, a * NE + n, f0);
                if (++st == kRStages) { st = 0; ph ^= 1; }
            }
        }
        __syncwarp();
    } else if (warp == 1) {
        // ------------------------------------------------------- MMAs
        if (lane == 0) {
            uint32_t rs = 0, rph = 0, ws = 0, wph = 0;
            bool first = true;
            for (int q = 0; q < npairs && !*s_abort; ++q) {
                const int e = s_tab[q];
                const bool ok = mbar_wait(&full_w[ws], wph, &g_das_tc_wait_error, 302) &&
                                mbar_wait(&full_r[rs], rph, &g_das_tc_wait_error, 303);
                if (!ok) {
                    *s_abort = 1;
                    break;
                }
                tc_fence_after();
                const int steps = e & 7;
                const uint32_t wa = smem_u32(sW + ws * kWBytes), ra = smem_u32(sR + rs * RB);
                for (int kk = 0; kk < steps; ++kk) {
                    mma_f16(tmem, desc_sw128_kmajor(wa) + 2 * kk, desc_sw128_kmajor(ra) + 2 * kk,
                            idesc, first ? 0u : 1u);
                    first = false;
                }
                mma_commit(&empty_w[ws]);
                mma_commit(&empty_r[rs]);
                if (++ws == kWStages) { ws = 0; wph ^= 1; }
                if (++rs == kRStages) { rs = 0; rph ^= 1; }
            }
            mma_commit(done);
        }
        __syncwarp();
    } else {
        // ------------ weight tiles, one pixel per thread; two groups of four
        // warps take alternate pairs (stages g and g + 2 of the ring)
        const int grp = (warp - 2) >> 2;
        const int m = 32 * (warp & 3) + lane;  // tensor-memory lane = pixel row of W
        const int col = m % kTX;
        const int ix = tx * kTX + col, iz = tz * kTZ + m / kTX;
        const bool valid = ix < d.nx && iz < d.nz;
        const int ixc = valid ? ix : 0, izc = valid ? iz : 0;
        const float zs = __ldg(d.zs + izc);
        if (grp == 0) {
            for (int a = 0; a < A; ++a) {
                const int bi = __ldg(d.bxi + a * d.nx + ixc) + __ldg(d.bzi + a * d.nz + izc);
                const float bf = __ldg(d.bxf + a * d.nx + ixc) + __ldg(d.bzf + a * d.nz + izc);
                s_base[a * kM + m] = make_int2(bi, __float_as_int(bf));
            }
        }
        asm volatile("bar.sync 1, 256;" ::: "memory");  // both groups read s_base
        uint8_t* const rowp = sW + (m >> 3) * 1024 + (m & 7) * 128;
        const int swz = m & 7;
        float w = 0.f, exc = 0.f;
        int cur_n = -1;
        int n = n_lo + grp / A, a = grp % A;
        // lateral offset of the group's next element, loaded one element ahead
        // (a single-angle plan gives each group every other element)
        int pre_n = n;
        float dxs_next = n <= n_hi ? __ldg(d.dxs + (size_t)n * d.nx + ixc) : 0.f;
        for (int q = grp; q < npairs && !*s_abort; q += 2) {
            if (n != cur_n) {
                cur_n = n;
                const float dxs = n == pre_n ? dxs_next : __ldg(d.dxs + (size_t)n * d.nx + ixc);
                pre_n = n + (A == 1 ? 2 : 1);
                if (pre_n <= n_hi) dxs_next = __ldg(d.dxs + (size_t)pre_n * d.nx + ixc);
                w = valid ? apod_weight(dxs, zs, d.fnum) : 0.f;
                exc = rx_excess(dxs, zs);
            }
            const int st = q & (kWStages - 1);
            const uint32_t ph = (uint32_t)(q / kWStages) & 1u;
            const int e = s_tab[q];
            const int k0 = e >> 3, lim = (e & 7) * 16;
            if (!mbar_wait(&empty_w[st], ph ^ 1u, &g_das_tc_wait_error, 304)) {
                *s_abort = 1;
                break;
            }
            uint8_t* W = rowp + st * kWBytes;
            const int pc = prev[st * kM + m];
            if (pc >= 0) {
                *reinterpret_cast<uint4*>(W + ((((pc >> 3)) ^ swz) << 4)) = make_uint4(0, 0, 0, 0);
                if ((pc & 7) > 4)
                    *reinterpret_cast<uint4*>(W + ((((pc >> 3) + 1) ^ swz) << 4)) =
                        make_uint4(0, 0, 0, 0);
            }
            int nc = -1;
            if (w != 0.f) {
                const int2 bs = s_base[a * kM + m];
                const float uf = __int_as_float(bs.y) + exc;
                const float fl = floorf(uf);
                const float phi = uf - fl;
                const int i = bs.x + (int)fl;
                float v[4];
                int c;
                if (d.interp == TIDAS_INTERP_CUBIC) {
                    keys_weights(phi, v[0], v[1], v[2], v[3]);
                    c = i - 1 - k0;
                } else {
                    v[0] = 1.f - phi;
                    v[1] = phi;
                    v[2] = 0.f;
                    v[3] = 0.f;
                    c = i - k0;
                }
                if (c >= 0 && c + 3 < lim) {  // always true by the table's construction
                    const __half2 h01 = __floats2half2_rn(w * v[0], w * v[1]);
                    const __half2 h23 = __floats2half2_rn(w * v[2], w * v[3]);
                    const uint64_t pk = (uint64_t)*reinterpret_cast<const uint32_t*>(&h01) |
                                        ((uint64_t)*reinterpret_cast<const uint32_t*>(&h23) << 32);
                    uint4 lo, hi;
                    place4(pk, c & 7, lo, hi);
                    *reinterpret_cast<uint4*>(W + (((c >> 3) ^ swz) << 4)) = lo;
                    if ((c & 7) > 4) *reinterpret_cast<uint4*>(W + ((((c >> 3) + 1) ^ swz) << 4)) = hi;
                    nc = c;
                }
            }
            prev[st * kM + m] = nc;
            fence_proxy_async_smem();
            __syncwarp();
            if (lane == 0) mbar_arrive(&full_w[st]);
            a += 2;
            while (a >= A) {
                a -= A;
                ++n;
            }
        }
        if (grp == 0) {  // epilogue: the first group holds every tensor-memory lane
        // --------------------------------------------------- epilogue
        bool have = npairs > 0;
        if (have && !mbar_wait(done, 0, &g_das_tc_wait_error, 305)) {
            *s_abort = 1;
            have = false;
        }
        tc_fence_after();
        const size_t plane = (size_t)d.nz * d.nx;
        for (int j = 0; j < NF; j += 32) {
            uint32_t r[32];
            if (have && !*s_abort) {
                tmem_ld_32x32b_x32(tmem + ((uint32_t)(32 * (warp & 3)) << 16) + (uint32_t)j, r);
                tmem_ld_wait();
            } else {
#pragma unroll
                for (int e2 = 0; e2 < 32; ++e2) r[e2] = 0u;
            }
            if (valid) {
                float* dst = img + (size_t)(f0 + j) * plane + (size_t)iz * d.nx + ix;
#pragma unroll
                for (int e2 = 0; e2 < 32; ++e2)
                    if (f0 + j + e2 < nf && j + e2 < NF) dst[(size_t)e2 * plane] = __uint_as_float(r[e2]);
            }
        }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
}

int make_map_3d(CUtensorMap* map, const void* ptr, CUtensorMapDataType dt, int esize, int nz,
                int nx, int nf, int box_x, int box_f, CUtensorMapSwizzle sw);

// Build the window table of an FP16 plan (once, at plan creation).
int das_tc_prepare(Plan& P) {
    const DasDev& d = P.dev;
    P.tc_tiles_x = (d.nx + dtc::kTX - 1) / dtc::kTX;
    P.tc_tiles = P.tc_tiles_x * ((d.nz + dtc::kTZ - 1) / dtc::kTZ);
    const size_t ntab = (size_t)P.tc_tiles * d.n_angles * d.n_elem;
    P.tc_ok = false;
    void* buf = nullptr;
    TIDAS_CUDA(cudaMalloc(&buf, ntab * 4 + (size_t)P.tc_tiles * 8 + 512));
    P.tc_tab = (int*)buf;
    P.tc_range = (int2*)((char*)buf + ((ntab * 4 + 255) & ~(size_t)255));
    int* d_bad = (int*)((char*)P.tc_range + P.tc_tiles * 8);
    std::vector<int2> init(P.tc_tiles, make_int2(INT_MAX, INT_MIN));
    TIDAS_CUDA(cudaMemcpy(P.tc_range, init.data(), P.tc_tiles * 8, cudaMemcpyHostToDevice));
    TIDAS_CUDA(cudaMemset(d_bad, 0, 4));
    long long blocks = ((long long)ntab + 255) / 256;
    das_tc_table_kernel<<<(int)(blocks > 152 * 64 ? 152 * 64 : blocks), 256>>>(
        d, P.tc_tiles_x, P.tc_tiles, P.tc_tab, P.tc_range, d_bad);
    int rc = check_launch("das_tc_table_kernel");
    if (rc) return rc;
    int bad = 0;
    TIDAS_CUDA(cudaMemcpy(&bad, d_bad, 4, cudaMemcpyDeviceToHost));
    P.tc_ok = (bad == 0) && dtc::smem_bytes(16, d.n_angles, d.n_elem) <= 227 * 1024;
    return TIDAS_OK;
}

int launch_das_tc(const Plan& P, const void* rf, float* img, int nf, cudaStream_t st) {
    using namespace dtc;
    const DasDev& d = P.dev;
    // the widest frame tile (MMA N) that the batch fills and shared memory holds
    int NF = 16;
    for (int c = 128; c > 16; c /= 2)
        if (nf >= c && smem_bytes(c, d.n_angles, d.n_elem) <= 227 * 1024) {
            NF = c;
            break;
        }
    CUtensorMap map;
    // channel data as [frames][angles * elements][samples]: box 64 samples x 1 row x NF frames
    int rc = make_map_3d(&map, rf, CU_TENSOR_MAP_DATA_TYPE_FLOAT16, 2, d.n_angles * d.n_elem,
                         d.n_samples, nf, kKW, NF, CU_TENSOR_MAP_SWIZZLE_128B);
    if (rc) return rc;
    const size_t smem = smem_bytes(NF, d.n_angles, d.n_elem);
    cudaFuncSetAttribute(das_tc_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    dim3 grid(P.tc_tiles, (nf + NF - 1) / NF);
    das_tc_kernel<<<grid, 320, smem, st>>>(map, d, P.tc_tab, P.tc_range, P.tc_tiles_x, nf, NF,
                                           img);
    return check_launch("das_tc_kernel");
}

}  // namespace tidas
