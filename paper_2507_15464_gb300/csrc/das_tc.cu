// Delay and Sum (Eq. (2.2)) for batches of FP16 channel data on the tcgen05
// tensor cores.
//
// For a tile of 128 pixels (32 columns x 4 rows) and a tile of NF frames,
//     img[p, f] = sum_{a,n} sum_k W_an[p, k] * rf[f, a, n, k0_an + k],
// where row p of W_an holds the apodized interpolation weights
// w_n(p) * K(u - m) of the (2 or 4) samples m that pixel p reads, placed at
// columns m - k0_an.  Over one tile every (angle, element) pair reads fewer
// than 64 consecutive samples, so each pair is a dense 128 x NF x (16 s)
// FP16 contraction (s = 1..4 K-steps) accumulated in FP32 tensor memory.  The
// window start k0_an (a multiple of 8) and s are tabulated per (tile, angle,
// element) when the plan is created.
//
// Channel data.  A TMA box of NF frames x 64 samples is NF separate rows of
// the [frame][angle, element][sample] layout, and the copy engine spends
// about as long on a row as on a kilobyte of contiguous data.  So each batch
// is first repacked (das_tc_pack_kernel, one HBM-bound pass) into
// [frame tile][angle, element][sample][NF frames] with the 16-byte chunks of
// every sample row already permuted into the MMA's swizzled MN-major operand
// layout, and 64 zero samples before and after each record.  The s K-steps
// of a pair are then s x 16 consecutive sample rows, one contiguous
// cp.async.bulk copy.
//
// Warp roles (12 warps, two groups):
//  - warps 0, 1: producers of group 0 / group 1: one bulk copy per pair into
//    the group's ring of K-step chunks (as many rounds in flight as the ring
//    holds).  Warp 0 also owns tensor memory.
//  - warps 2-5 / 6-9: the builders of group 0 / group 1.  The pairs of a
//    tile are cut into rounds of one or two consecutive pairs whose K-steps
//    fit one 64-column weight tile together (at plan creation, greedily from
//    the first pair), and the groups take alternate rounds.  Every thread
//    owns one pixel (one row of W_an, one tensor-memory lane): it erases the
//    8-byte words it wrote two rounds ago and writes each pair's four weights
//    as the one or two 8-byte words they cover in its row of a 128-byte-
//    swizzled K-major weight tile (two per group), the second pair's columns
//    after the first's.
//  - warps 10, 11: the MMA warps of group 0 / group 1.  Builders and MMA warp
//    meet at a named barrier once per round; then the MMA warp issues the
//    round's K-steps into the group's own accumulator while the builders write
//    the next round, and one tcgen05.commit per round frees both the weight
//    tile and the round's chunks.  A single thread issues one tcgen05.mma about
//    every 100 cycles, while a 128 x 64 x 16 step occupies the tensor pipe
//    for about 50, so two issuing threads per CTA (four per SM) keep it fed.
//    Merging pairs into rounds (0.63 rounds per pair on the 128-element,
//    11-angle grid) saves a barrier, a commit and the loop bookkeeping of
//    every merged pair.
// The epilogue sums the two accumulators.
#include <climits>
#include <mutex>
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
constexpr int kTX = 32, kTZ = 4;          // pixel tile: one row of 32 per warp
constexpr int kM = kTX * kTZ;             // 128 = UMMA M
constexpr int kKW = 64;                   // weight-tile columns (one 128-byte swizzle row)
constexpr int kKC = 16;                   // samples per K-step chunk
constexpr int kMaxSteps = kKW / kKC;
constexpr int kPad = 64;                  // zero samples before and after each packed record
constexpr int kPackS = 64;                // samples per pack block
constexpr int kGroups = 2;                // builder groups, one accumulator each
constexpr int kWTiles = 2 * kGroups;      // weight tiles: two per group
constexpr int kWBytes = kM * kKW * 2;     // 16 KB
constexpr int kPairSlots = 8;             // rounds of a group in flight (barrier slots)
// Window entry, 16 bits: 2 * k0 + K-steps (0..4); k0 is a multiple of 8 in
// [-kMaxK0, kMaxK0].
constexpr int kMaxK0 = 16376;
__host__ __device__ constexpr int entry_k0(int e) { return (e >> 4) * 8; }
// Round descriptor, 8 bits: the round's K-steps (0..4) + kTwoPairs if it
// holds two pairs.
constexpr int kTwoPairs = 8;
__host__ __device__ constexpr int round_pairs(int rd) { return 1 + (rd >> 3); }
constexpr int kMinChunks = 6, kMaxChunks = 32;  // chunks per group ring
// per group: one producer warp, four builder warps, one MMA warp
constexpr int kBuilderWarp0 = kGroups;            // warps [0, kGroups): producers
constexpr int kMmaWarp0 = kGroups + 4 * kGroups;  // warps [kMmaWarp0, kWarps): MMA warps
constexpr int kWarps = kMmaWarp0 + kGroups;
constexpr int kThreads = 32 * kWarps;
static_assert(kWarps == 6 * kGroups && kGroups == 2, "warp roles assume two groups of six warps");
constexpr int kEpiBarCount = 32 * 5 * kGroups;    // builders wait, MMA warps arrive
constexpr size_t kSmemTwoPerSM = 115712;  // (228 KB - 2 x 1 KB reserved) / 2
constexpr size_t kSmemMax = 227 * 1024;
// one K-step chunk = 16 sample rows of NF frames
__host__ __device__ constexpr int chunk_bytes(int NF) { return kKC * NF * 2; }
// align | weight tiles | chunk rings | barriers, flags (512 B) |
// transmit split [A][kM] int2 | window entries [A * NE] int16 |
// round descriptors [A * NE] uint8 (a tile has at most one round per pair)
constexpr size_t kFlagBytes = 512;
__host__ __device__ constexpr size_t fixed_bytes(int A, int NE) {
    return 1024 + (size_t)kWTiles * kWBytes + kFlagBytes + (size_t)A * kM * 8 +
           (((size_t)A * NE * 2 + 15) & ~(size_t)15) + (((size_t)A * NE + 15) & ~(size_t)15);
}
__host__ __device__ constexpr size_t smem_bytes(int NF, int C, int A, int NE) {
    return fixed_bytes(A, NE) + (size_t)kGroups * C * chunk_bytes(NF);
}
// packed record length (samples, margins included)
__host__ __device__ constexpr int packed_len(int S) {
    return (S + kPackS - 1) / kPackS * kPackS + 2 * kPad;
}
}  // namespace dtc

// Swizzled position of 16-byte chunk c in sample row k of an MN-major operand
// whose rows hold NF frames (NF * 2 bytes): the 128-, 64- or 32-byte swizzle
// XORs the chunk index with bits of the row index (address bits 7.. into
// bits 4..), repeating every 8 rows.
__host__ __device__ __forceinline__ int mn_swizzle(int c, int k, int NF) {
    return NF == 64 ? c ^ (k & 7) : NF == 32 ? c ^ ((k >> 1) & 3) : c ^ ((k >> 2) & 1);
}

// [nf][R][S] FP16 -> [FT][R][Sp][NF] FP16, sample s at s + kPad, frames past
// nf and samples outside [0, S) or outside the read window [rd_lo, rd_hi)
// zero, chunks swizzled (mn_swizzle).  One block per (frame
// tile, row, 64-sample block sb_first .. sb_first + nbw - 1); S is a
// multiple of 8.
//
// The transpose goes through shared memory as 32-bit words, each holding one
// sample of two neighbouring frames.  Sample row r keeps its NF / 8 chunks of
// 16 bytes with the chunk index XORed with (r / 8) mod (NF / 8): at NF = 64
// the word stores of a warp (8 sample rows x 4 frame pairs) and the chunk
// loads that follow both touch every bank once per wavefront.
__global__ void __launch_bounds__(256) das_tc_pack_kernel(const __half* __restrict__ rf,
                                                          __half* __restrict__ out, int nf, int R,
                                                          int S, int Sp, int NF, int sb_first,
                                                          int nbw, int rd_lo, int rd_hi) {
    using namespace dtc;
    __shared__ uint4 tile[kPackS * 8];  // [kPackS rows][NF / 8 chunks]
    const int cpr = NF / 8;             // chunks per sample row (2, 4 or 8)
    const int sb = sb_first + (int)(blockIdx.x % nbw);
    const int row = (blockIdx.x / nbw) % R;
    const int ft = blockIdx.x / (nbw * R);
    const int s0 = sb * kPackS - kPad;
    uint32_t* t32 = reinterpret_cast<uint32_t*>(tile);
    // load frame pairs x 64 samples as 16-byte chunks of 8 samples
    for (int i = threadIdx.x; i < (NF / 2) * (kPackS / 8); i += blockDim.x) {
        const int c = i % (kPackS / 8), fp = i / (kPackS / 8);
        const int s = s0 + 8 * c, fa = ft * NF + 2 * fp;
        uint4 va = make_uint4(0, 0, 0, 0), vb = make_uint4(0, 0, 0, 0);
        if (s >= 0 && s < S && s + 8 > rd_lo && s < rd_hi) {
            if (fa < nf)
                va = __ldg(reinterpret_cast<const uint4*>(rf + ((size_t)fa * R + row) * S + s));
            if (fa + 1 < nf)
                vb = __ldg(
                    reinterpret_cast<const uint4*>(rf + ((size_t)(fa + 1) * R + row) * S + s));
        }
        uint32_t a[4] = {va.x, va.y, va.z, va.w}, b[4] = {vb.x, vb.y, vb.z, vb.w};
        if (s < rd_lo || s + 8 > rd_hi) {
            // a chunk across an end of the window: its samples outside are zero
#pragma unroll
            for (int t = 0; t < 4; ++t) {
                const uint32_t keep = (s + 2 * t >= rd_lo && s + 2 * t < rd_hi ? 0x0000FFFFu : 0u) |
                                      (s + 2 * t + 1 >= rd_lo && s + 2 * t + 1 < rd_hi ? 0xFFFF0000u : 0u);
                a[t] &= keep;
                b[t] &= keep;
            }
        }
#pragma unroll
        for (int t = 0; t < 4; ++t) {
            const int r0 = 8 * c + 2 * t;  // rows r0, r0 + 1 share r / 8
            const int w = 4 * cpr * r0 + 4 * ((fp >> 2) ^ ((r0 >> 3) & (cpr - 1))) + (fp & 3);
            t32[w] = __byte_perm(a[t], b[t], 0x5410);            // sample r0: frames fa, fa + 1
            t32[w + 4 * cpr] = __byte_perm(a[t], b[t], 0x7632);  // sample r0 + 1
        }
    }
    __syncthreads();
    // store 64 sample rows of NF frames, 16-byte chunks swizzled
    __half* dst = out + (((size_t)ft * R + row) * Sp + (size_t)sb * kPackS) * NF;
    for (int i = threadIdx.x; i < kPackS * cpr; i += blockDim.x) {
        const int k = i / cpr, c = i % cpr;
        *reinterpret_cast<uint4*>(dst + (size_t)k * NF + 8 * mn_swizzle(c, k, NF)) =
            tile[k * cpr + (c ^ ((k >> 3) & (cpr - 1)))];
    }
}

// Shared-memory descriptor of one MN-major K-step chunk (16 sample rows of NF
// frames) in the swizzle matching NF (64: 128-byte, 32: 64-byte, 16: 32-byte):
// a single swizzle atom spans the MN extent, atoms of 8 rows follow along K.
// Both byte-offset fields carry the 8-row stride; with one atom along MN only
// the K-direction stride is read.
__device__ __forceinline__ uint64_t desc_mn_chunk(uint32_t smem_addr, int NF) {
    const uint64_t stride = (uint64_t)(8 * NF * 2) >> 4;
    const uint64_t layout = NF == 64 ? 2 : NF == 32 ? 4 : 6;
    return (uint64_t)((smem_addr & 0x3FFFFu) >> 4) | (stride << 16) | (stride << 32) |
           ((uint64_t)1 << 46) | (layout << 61);
}

// The 8-byte word of a weight-tile row that holds column c (0..63): byte
// 2 c rounded down to 8, with the 16-byte chunk index (bits 4..6) XORed with
// the row's swizzle; swz16 = swizzle << 4.
__device__ __forceinline__ uint64_t* row_word(uint8_t* row, int c, int swz16) {
    return reinterpret_cast<uint64_t*>(row + (((c << 1) & 0x78) ^ swz16));
}

// Hand-off between group g's 128 builders and its MMA warp (160 threads):
// a barrier that both sides wait on, once per round, which also tells every
// participant whether any of them has given up.  While the builders write
// round j + 1 the MMA warp issues round j, so the two overlap.
__device__ __forceinline__ bool group_bar(int grp, int stop) {
    constexpr int kCount = 32 * 5;
    return grp == 0 ? named_bar_or<2>(kCount, stop) : named_bar_or<3>(kCount, stop);
}

// Hann apodization of one (pixel, element) for the weight builders: the zero
// cut |r| > 1/2 is decided by the same operations as in the window table,
// and inside it the fast cosine intrinsic (absolute error about 5e-7) stands
// in for cospif, far below the FP16 rounding of the weights (2^-11).
__device__ __forceinline__ float builder_apod(float dxs, float zs, float fnum) {
    if (fnum <= 0.f) return 1.f;
    const float r = dxs * fnum / zs;
    if (fabsf(r) > 0.5f) return 0.f;
    const float cw = __cosf(3.14159265358979f * r);
    return cw * cw;
}

// First pair of a group's next round, after its round r of `len` pairs that
// starts at pair q: the other group's round r + 1 comes in between (rounds
// alternate between the groups).  npairs or more when there is none.
__device__ __forceinline__ int next_round(const uint8_t* s_rd, int r, int q, int len,
                                          int npairs) {
    const int q1 = q + len;
    return q1 < npairs ? q1 + dtc::round_pairs(s_rd[r + 1]) : q1;
}

// Per-(tile, angle, element) window: entry = 2 k0 + ksteps, k0 a multiple of
// 8 and ksteps in 0..4 (0: no contributing pixel, or a window wholly outside
// the record, whose samples are all zero; k0 is then 0).  Per tile: the range
// of contributing elements.
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
            int k0 = (int)floorf((float)c_lo / 8.f) * 8;
            const int span = c_hi - k0 + 1;
            int steps = (span + dtc::kKC - 1) / dtc::kKC;
            if (steps > dtc::kMaxSteps) atomicExch(bad, 1);
            steps = min(steps, dtc::kMaxSteps);
            // a window that misses [0, n_samples) reads only zeros; any other
            // one lies inside the packed record's zero margins
            if (k0 + dtc::kKC * steps <= 0 || k0 >= d.n_samples) {
                steps = 0;
                k0 = 0;
            }
            // the kernel keeps a 16-bit copy of the entry in shared memory
            if (k0 < -dtc::kMaxK0 || k0 > dtc::kMaxK0) atomicExch(bad, 1);
            entry = 2 * k0 + steps;
            atomicMin(&range[tile].x, n);
            atomicMax(&range[tile].y, n);
        }
        tab[q] = entry;
    }
}

template <int INTERP>
__global__ void __launch_bounds__(dtc::kThreads, 2)
    das_tc_kernel(const __half* __restrict__ packed, DasDev d, const int* __restrict__ tab,
                  const int2* __restrict__ range, const uint8_t* __restrict__ rounds,
                  int tiles_x, int nf, int NF, int C, float* __restrict__ img) {
    using namespace dtc;
    extern __shared__ uint8_t smem_raw[];
    uint8_t* base = smem_align1024(smem_raw);
    const int CB = chunk_bytes(NF);
    const int A = d.n_angles, NE = d.n_elem;
    const int Sp = packed_len(d.n_samples);
    uint8_t* sW = base;                                        // [kWTiles] weight tiles
    uint8_t* sC = base + kWTiles * kWBytes;                    // [kGroups][C] chunks
    // group g, round slot p: full completes when the round's chunks have
    // landed, empty when its MMAs have finished reading its chunks and tile
    uint64_t* full = (uint64_t*)(sC + kGroups * C * CB);      // [kGroups][kPairSlots]
    uint64_t* empty = full + kGroups * kPairSlots;             // [kGroups][kPairSlots]
    uint64_t* done = empty + kGroups * kPairSlots;             // [kGroups]
    uint32_t* tmem_slot = (uint32_t*)(done + kGroups);
    volatile int* s_abort = (volatile int*)(tmem_slot + 1);
    int* s_used = (int*)(tmem_slot + 2);                       // [kGroups]
    int2* s_base = (int2*)((uint8_t*)full + kFlagBytes);       // [A][kM]: transmit split
    int16_t* s_tab = (int16_t*)(s_base + A * kM);              // [pair]: window entries
    uint8_t* s_rd = (uint8_t*)s_tab + (((size_t)A * NE * 2 + 15) & ~(size_t)15);  // [round]

    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    // deepest tiles first: their apertures span the most elements, so the
    // last wave of CTAs holds the cheap shallow tiles and the tail stays short
    const int tile = gridDim.x - 1 - blockIdx.x;
    const int tx = tile % tiles_x, tz = tile / tiles_x;
    const int f0 = blockIdx.y * NF;
    const int2 rg = range[tile];
    const int n_lo = rg.x, n_hi = rg.y;
    const int npairs = n_hi >= n_lo ? (n_hi - n_lo + 1) * A : 0;
    const uint32_t acc_cols = NF < 32 ? 32 : NF;              // columns per accumulator
    const uint32_t tcols = kGroups * acc_cols;

    if (threadIdx.x == 0) {
        for (int s = 0; s < kGroups * kPairSlots; ++s) {
            mbar_init(&full[s], 1);
            mbar_init(&empty[s], 1);
        }
        for (int g = 0; g < kGroups; ++g) {
            mbar_init(&done[g], 1);
            s_used[g] = 0;
        }
        *s_abort = 0;
        fence_barrier_init();
    }
    // zero the weight tiles once; afterwards only written words are erased
    for (int i = threadIdx.x; i < kWTiles * kWBytes / 16; i += blockDim.x)
        reinterpret_cast<uint4*>(sW)[i] = make_uint4(0, 0, 0, 0);
    // this tile's window entries (pair order: element-major, angle-minor) and
    // the transmit split of its pixels, so that no role waits on a global load
    // per pair
    {
        const int* tt = tab + (size_t)tile * A * NE;
        const uint8_t* tr = rounds + (size_t)tile * A * NE;
        for (int i = threadIdx.x; i < npairs; i += blockDim.x) {
            s_tab[i] = (int16_t)__ldg(tt + (i % A) * NE + n_lo + i / A);
            s_rd[i] = __ldg(tr + i);
        }
        for (int i = threadIdx.x; i < A * kM; i += blockDim.x) {
            const int a = i / kM, m = i % kM;
            const int ix = tx * kTX + m % kTX, iz = tz * kTZ + m / kTX;
            const int ixc = ix < d.nx ? ix : 0, izc = iz < d.nz ? iz : 0;
            const int bi = __ldg(d.bxi + a * d.nx + ixc) + __ldg(d.bzi + a * d.nz + izc);
            const float bf = __ldg(d.bxf + a * d.nx + ixc) + __ldg(d.bzf + a * d.nz + izc);
            s_base[i] = make_int2(bi, __float_as_int(bf));
        }
    }
    if (warp == 0) {
        tmem_alloc(tmem_slot, tcols);
        tmem_relinquish();
    }
    fence_proxy_async_smem();
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp < kBuilderWarp0) {
        // ------------------- producer of group g: the K-steps of its pairs
        const int grp = warp;
        if (lane == 0) {
            uint64_t* gfull = full + grp * kPairSlots;
            uint64_t* gempty = empty + grp * kPairSlots;
            uint8_t* ring = sC + grp * C * CB;
            const __half* src_tile = packed + (size_t)blockIdx.y * A * NE * Sp * NF;
            int head = 0, free_chunks = C, oldest = 0, j = 0;
            int qa = 0, n = n_lo, a = 0;  // pair qa is (element n, angle a)
            uint32_t pend = 0;            // K-steps of the rounds in flight, 3 bits per slot
            bool bad = false;
            // global round r = 2 j + grp starts at pair q
            int q = grp == 0 || npairs == 0 ? 0 : round_pairs(s_rd[0]);
            for (int len; q < npairs && !bad;
                 q = next_round(s_rd, 2 * j + grp, q, len, npairs), ++j) {
                const int rd = s_rd[2 * j + grp];
                len = round_pairs(rd);
                const int steps = rd & 7;
                const int e0 = s_tab[q], e1 = len == 2 ? s_tab[q + 1] : 0;
                // reuse of the round slot, and room for this round's chunks:
                // retire the oldest rounds in flight
                while (!bad && oldest < j && (oldest <= j - kPairSlots || free_chunks < steps)) {
                    if (!mbar_wait_or_abort(&gempty[oldest % kPairSlots],
                                            (uint32_t)(oldest / kPairSlots) & 1u, s_abort,
                                            &g_das_tc_wait_error, 301)) {
                        bad = true;
                        break;
                    }
                    free_chunks += (int)(pend >> (3 * (oldest % kPairSlots))) & 7;
                    ++oldest;
                }
                if (bad) break;
                const int sh = 3 * (j % kPairSlots);
                pend = (pend & ~(7u << sh)) | ((uint32_t)steps << sh);
                uint64_t* bar = &gfull[j % kPairSlots];
                mbar_arrive_expect_tx(bar, (uint32_t)(steps * CB));
                for (int p = 0; p < len; ++p) {
                    a += q + p - qa;
                    qa = q + p;
                    while (a >= A) {
                        a -= A;
                        ++n;
                    }
                    const int e = p ? e1 : e0;
                    const int sp = e & 7;
                    if (sp) {
                        // sample rows k0 .. k0 + 16 sp of row (a, n): contiguous
                        const uint8_t* src = reinterpret_cast<const uint8_t*>(
                            src_tile + ((size_t)(a * NE + n) * Sp + (size_t)(entry_k0(e) + kPad)) * NF);
                        const int first = sp <= C - head ? sp : C - head;
                        bulk_load(ring + head * CB, src, (uint32_t)(first * CB), bar);
                        if (first < sp)
                            bulk_load(ring, src + (size_t)first * CB, (uint32_t)((sp - first) * CB),
                                      bar);
                    }
                    head += sp;
                    if (head >= C) head -= C;
                }
                free_chunks -= steps;
            }
            if (*s_abort) {
                // the consumers gave up: let the copies still in flight land
                // before the CTA's shared memory is released
                for (int k = 1; k <= kPairSlots && j - k >= oldest; ++k) {
                    const int jj = j - k;
                    mbar_wait(&gfull[jj % kPairSlots], (uint32_t)(jj / kPairSlots) & 1u,
                              &g_das_tc_wait_error, 306);
                }
            }
        }
        __syncwarp();
    } else if (warp >= kMmaWarp0) {
        // ------------------------------------------ MMA warp of group g
        const int grp = warp - kMmaWarp0;
        const uint32_t acc = tmem + (uint32_t)grp * acc_cols;
        const uint32_t idesc = idesc_f16_f32(kM, NF) | (1u << 16);  // B is MN-major
        uint64_t* gfull = full + grp * kPairSlots;
        uint64_t* gempty = empty + grp * kPairSlots;
        const uint32_t ring = smem_u32(sC + grp * C * CB);
        int pos = 0, j = 0;  // first chunk of round j in the ring
        bool bad = false;
        uint32_t accf = 0u;  // 0 until the group's first MMA has written its accumulator
        const uint64_t b0 = desc_mn_chunk(ring, NF);
        const uint32_t b_lo0 = (uint32_t)b0, b_hi = (uint32_t)(b0 >> 32);
        const uint32_t b_step = (uint32_t)CB >> 4, b_end = b_lo0 + (uint32_t)C * b_step;
        const uint64_t w0 = desc_sw128_kmajor(smem_u32(sW + grp * kWBytes));
        const uint32_t w_lo0 = (uint32_t)w0, w_hi = (uint32_t)(w0 >> 32);
        const uint32_t w_lo1 =
            (uint32_t)desc_sw128_kmajor(smem_u32(sW + (grp + kGroups) * kWBytes));
        int q = grp == 0 || npairs == 0 ? 0 : round_pairs(s_rd[0]);
        for (int len; q < npairs; q = next_round(s_rd, 2 * j + grp, q, len, npairs), ++j) {
            const int rd = s_rd[2 * j + grp];
            len = round_pairs(rd);
            // Round j - 1's MMAs must be complete before this barrier: past it the
            // builders write round j + 1 into the tile round j - 1 read.  (Its MMAs
            // ran while the builders wrote round j, so this rarely waits.)
            if (lane == 0 && j >= 1 && !bad)
                bad = !mbar_wait_or_abort(&gempty[(j - 1) % kPairSlots],
                                          (uint32_t)((j - 1) / kPairSlots) & 1u, s_abort,
                                          &g_das_tc_wait_error, 304);
            // the group's weight tile of round j is written (leave together on an abort)
            if (group_bar(grp, bad || *s_abort)) break;
            const int steps = rd & 7;
            if (lane == 0) {
                if (!bad && mbar_wait_or_abort(&gfull[j % kPairSlots],
                                               (uint32_t)(j / kPairSlots) & 1u, s_abort,
                                               &g_das_tc_wait_error, 303)) {
                    tc_fence_after();
                    // descriptors differ from the ring's first chunk and the
                    // weight tile's first K-step only in their start-address
                    // field (bits 0..13, shared address / 16), which the
                    // offsets below never carry out of
                    uint32_t wl = (j & 1) ? w_lo1 : w_lo0;
                    uint32_t bl = b_lo0 + (uint32_t)pos * b_step;
#pragma unroll
                    for (int kk = 0; kk < kKW / kKC; ++kk) {
                        if (kk < steps) {
                            mma_f16(acc, ((uint64_t)w_hi << 32) | wl, ((uint64_t)b_hi << 32) | bl,
                                    idesc, accf);
                            accf = 1u;
                            wl += 2;  // 32 bytes: the next 16 columns of the 128-byte rows
                            bl += b_step;
                            if (bl == b_end) bl = b_lo0;
                        }
                    }
                    mma_commit(&gempty[j % kPairSlots]);
                } else {
                    bad = true;
                }
            }
            pos += steps;
            if (pos >= C) pos -= C;
            __syncwarp();
        }
        if (lane == 0) {
            s_used[grp] = (int)accf;
            mma_commit(&done[grp]);  // arrives once this thread's MMAs have completed
        }
        __syncwarp();
        named_bar_arrive<1>(kEpiBarCount);
    } else {
        // ------------------- weight tiles, one pixel per thread; group g takes
        // rounds g, g + 2, ... into weight tiles g and g + 2
        const int grp = (warp - kBuilderWarp0) >> 2;
        const int m = 32 * (warp & 3) + lane;  // tensor-memory lane = pixel row of W
        const int ix = tx * kTX + m % kTX, iz = tz * kTZ + m / kTX;
        const bool valid = ix < d.nx && iz < d.nz;
        const int ixc = valid ? ix : 0, izc = valid ? iz : 0;
        const float zs = __ldg(d.zs + izc);
        uint8_t* const rowp = sW + (m >> 3) * 1024 + (m & 7) * 128;
        const int swz16 = (m & 7) << 4;
        float exc = 0.f;
        // apodized interpolation weights of element n as polynomials in the
        // fraction phi, with the Hann weight w folded into the coefficients
        // (Horner form): cubic Keys, w w0 = phi (phi (ca phi + cw) + ca),
        // w w1 = phi^2 (cc phi + cd) + cw, w w2 = phi (phi (cf - cc phi) + ch),
        // w w3 = phi^2 (ch phi - ch); linear w (1 - phi), w phi.  The cubic
        // coefficients are kept as the pairs that evaluate (w0, w2) and the
        // inner terms of (w1, w3) in packed instructions.
        float cw = 0.f;
        uint64_t k02a = 0, k02b = 0, k02c = 0, k13a = 0, k13b = 0;
        auto set_weight = [&](float w) {
            const float ca = -0.5f * w, cc = 1.5f * w, cd = -2.5f * w, cf = 2.f * w,
                        ch = 0.5f * w;
            cw = w;
            k02a = f2(ca, -cc);
            k02b = f2(w, cf);
            k02c = f2(ca, ch);
            k13a = f2(cc, ch);
            k13b = f2(cd, -ch);
        };
        // the column of the first tap this thread wrote into each of the
        // group's two tiles, per pair of the round that wrote it (-1: none):
        // r0 / r1 for the tile of the current round, o0 / o1 for the other
        int r0 = -1, r1 = -1, o0 = -1, o1 = -1;
        int n = n_lo, a = 0;  // at the top of a round: its first pair is (element n, angle a)
        // the lateral offset of element n + 1 is loaded one element ahead
        float dxs_next = 0.f;
        if (npairs > 0) {
            const float dxs = __ldg(d.dxs + (size_t)n * d.nx + ixc);
            set_weight(valid ? builder_apod(dxs, zs, d.fnum) : 0.f);
            exc = rx_excess(dxs, zs);
            if (n + 1 <= n_hi) dxs_next = __ldg(d.dxs + (size_t)(n + 1) * d.nx + ixc);
        }
        int j = 0;
        int q = grp == 0 || npairs == 0 ? 0 : round_pairs(s_rd[0]);
        a = q;
        for (; q < npairs; ++j) {
            const int len = round_pairs(s_rd[2 * j + grp]);
            // the tile was last read by this group's round j - 2, whose MMAs the
            // MMA warp saw complete before the previous group barrier
            {
                uint8_t* W = rowp + (grp + kGroups * (j & 1)) * kWBytes;
                if (r0 >= 0) {
                    *row_word(W, r0, swz16) = 0ull;
                    if (r0 & 3) *row_word(W, r0 + 4, swz16) = 0ull;
                }
                if (r1 >= 0) {
                    *row_word(W, r1, swz16) = 0ull;
                    if (r1 & 3) *row_word(W, r1 + 4, swz16) = 0ull;
                }
                r0 = -1;
                r1 = -1;
                int col0 = 0;  // first column of the pair in the weight tile
#pragma unroll
                for (int p = 0; p < 2; ++p) {
                    if (p == 1 && len == 1) break;
                    a += p;
                    if (a >= A) {
                        int dn = 0;
                        do {
                            a -= A;
                            ++n;
                            ++dn;
                        } while (a >= A);
                        const float dxs =
                            dn == 1 ? dxs_next : __ldg(d.dxs + (size_t)n * d.nx + ixc);
                        if (n + 1 <= n_hi) dxs_next = __ldg(d.dxs + (size_t)(n + 1) * d.nx + ixc);
                        set_weight(valid ? builder_apod(dxs, zs, d.fnum) : 0.f);
                        exc = rx_excess(dxs, zs);
                    }
                    const int e = s_tab[q + p];
                    const int k0 = entry_k0(e), steps = e & 7;
                    if (cw != 0.f) {
                        const int2 bs = s_base[a * kM + m];
                        const float uf = __int_as_float(bs.y) + exc;
                        const float fl = floorf(uf);
                        const float phi = uf - fl;
                        const int i = bs.x + (int)fl;
                        float v0, v1, v2, v3;
                        int c;
                        if (INTERP == TIDAS_INTERP_CUBIC) {
                            const float p2 = phi * phi;
                            const uint64_t P = f2(phi, phi);
                            const uint64_t t02 = f2_mul(f2_fma(f2_fma(k02a, P, k02b), P, k02c), P);
                            const uint64_t t13 = f2_fma(k13a, P, k13b);
                            v0 = f2_lo(t02);
                            v2 = f2_hi(t02);
                            v1 = fmaf(f2_lo(t13), p2, cw);
                            v3 = f2_hi(t13) * p2;
                            c = i - 1 - k0;
                        } else {
                            v0 = fmaf(-cw, phi, cw);
                            v1 = cw * phi;
                            v2 = 0.f;
                            v3 = 0.f;
                            c = i - k0;
                        }
                        // inside the pair's window by the table's construction,
                        // unless the window misses the record (steps 0)
                        if (c >= 0 && c + 3 < steps * kKC) {
                            const __half2 h01 = __floats2half2_rn(v0, v1);
                            const __half2 h23 = __floats2half2_rn(v2, v3);
                            const uint64_t pk =
                                (uint64_t)*reinterpret_cast<const uint32_t*>(&h01) |
                                ((uint64_t)*reinterpret_cast<const uint32_t*>(&h23) << 32);
                            // the taps' 8 bytes at half offset c of the row: one
                            // word, or the two words they straddle
                            c += col0;
                            const int sh = (c & 3) * 16;
                            *row_word(W, c, swz16) = pk << sh;
                            if (sh) *row_word(W, c + 4, swz16) = pk >> (64 - sh);
                            if (p)
                                r1 = c;
                            else
                                r0 = c;
                        }
                    }
                    col0 += steps * kKC;
                }
                // the next round writes the other tile
                const int t0 = r0, t1 = r1;
                r0 = o0;
                r1 = o1;
                o0 = t0;
                o1 = t1;
            }
            fence_proxy_async_smem();
            if (group_bar(grp, *s_abort)) break;
            // (n, a) of the first pair of the group's next round
            const int q2 = next_round(s_rd, 2 * j + grp, q, len, npairs);
            a += q2 - (q + len - 1);
            q = q2;
        }
        named_bar_sync<1>(kEpiBarCount);  // the MMA warps have committed `done`
        // --------------------------------------------------- epilogue: group g
        // drains the 32-column chunks j = g, g + 2, ... of both accumulators.
        // The waits are not cut short by an abort: MMAs still in flight must
        // finish before tensor memory is released.
        bool ok = true;
        for (int g = 0; g < kGroups; ++g)
            ok = mbar_wait(&done[g], 0, &g_das_tc_wait_error, 305) && ok;
        ok = ok && !*s_abort;
        tc_fence_after();
        const size_t plane = (size_t)d.nz * d.nx;
        const uint32_t lane_base = (uint32_t)(32 * (warp & 3)) << 16;
        for (int jc = 32 * grp; jc < NF; jc += 32 * kGroups) {
            float sum[32];
#pragma unroll
            for (int e2 = 0; e2 < 32; ++e2) sum[e2] = 0.f;
            for (int g = 0; g < kGroups; ++g) {
                if (!ok || !s_used[g]) continue;
                uint32_t r[32];
                tmem_ld_32x32b_x32(tmem + lane_base + (uint32_t)g * acc_cols + (uint32_t)jc, r);
                tmem_ld_wait();
#pragma unroll
                for (int e2 = 0; e2 < 32; ++e2) sum[e2] += __uint_as_float(r[e2]);
            }
            if (valid) {
                float* dst = img + (size_t)(f0 + jc) * plane + (size_t)iz * d.nx + ix;
#pragma unroll
                for (int e2 = 0; e2 < 32; ++e2)
                    if (f0 + jc + e2 < nf && jc + e2 < NF) dst[(size_t)e2 * plane] = sum[e2];
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, tcols);
    }
}

// Cut each tile's pairs (element-major, angle-minor, from its first
// contributing element) into rounds of one or two consecutive pairs,
// greedily from the first pair: a pair joins the round of the pair before it
// when that round holds one pair and their K-steps fit one weight tile.
// Round r of the tile is described by rounds[tile][r] (kTwoPairs + K-steps);
// a tile has at most one round per pair.  One thread per tile.
__global__ void das_tc_round_kernel(int A, int NE, int tiles, const int* __restrict__ tab,
                                    const int2* __restrict__ range,
                                    uint8_t* __restrict__ rounds) {
    const int tile = blockIdx.x * blockDim.x + threadIdx.x;
    if (tile >= tiles) return;
    const int2 rg = range[tile];
    if (rg.y < rg.x) return;
    const int npairs = (rg.y - rg.x + 1) * A;
    const int* tt = tab + (size_t)tile * A * NE + rg.x;
    uint8_t* out = rounds + (size_t)tile * A * NE;
    int r = 0;
    for (int q = 0; q < npairs;) {
        // pair q is (element rg.x + q / A, angle q % A)
        const int s0 = tt[(q % A) * NE + q / A] & 7;
        const int s1 = q + 1 < npairs ? tt[((q + 1) % A) * NE + (q + 1) / A] & 7 : dtc::kMaxSteps + 1;
        if (s0 + s1 <= dtc::kMaxSteps) {
            out[r++] = (uint8_t)(dtc::kTwoPairs + s0 + s1);
            q += 2;
        } else {
            out[r++] = (uint8_t)s0;
            q += 1;
        }
    }
}

// The plan's staging buffer of das_forward (the repacked batch of either DAS
// path), grown to `need` bytes on demand.  cudaFree / cudaMalloc synchronise
// the device, which is why das_forward calls on one plan must not overlap.
int plan_staging(const Plan& P, size_t need, void** out, long long layout, bool* fresh) {
    std::lock_guard<std::mutex> lock(P.tc_ws_mutex);
    if (need > P.tc_ws_bytes) {
        P.tc_ws_layout = 0;
        if (P.tc_ws) TIDAS_CUDA(cudaFree(P.tc_ws));
        P.tc_ws = nullptr;
        P.tc_ws_bytes = 0;
        TIDAS_CUDA(cudaMalloc(&P.tc_ws, need));
        P.tc_ws_bytes = need;
    }
    *fresh = P.tc_ws_layout != layout;
    P.tc_ws_layout = layout;
    *out = P.tc_ws;
    return TIDAS_OK;
}

// Build the window table of an FP16 plan (once, at plan creation).
int das_tc_prepare(Plan& P) {
    const DasDev& d = P.dev;
    P.tc_tiles_x = (d.nx + dtc::kTX - 1) / dtc::kTX;
    P.tc_tiles = P.tc_tiles_x * ((d.nz + dtc::kTZ - 1) / dtc::kTZ);
    const size_t ntab = (size_t)P.tc_tiles * d.n_angles * d.n_elem;
    P.tc_ok = false;
    void* buf = nullptr;
    // window entries | per-tile element range | round descriptors | flag
    const size_t off_range = (ntab * 4 + 255) & ~(size_t)255;
    const size_t off_rounds = (off_range + (size_t)P.tc_tiles * 8 + 255) & ~(size_t)255;
    const size_t off_bad = (off_rounds + ntab + 255) & ~(size_t)255;
    TIDAS_CUDA(cudaMalloc(&buf, off_bad + 256));
    P.tc_tab = (int*)buf;
    P.tc_range = (int2*)((char*)buf + off_range);
    P.tc_rounds = (uint8_t*)buf + off_rounds;
    int* d_bad = (int*)((char*)buf + off_bad);
    TIDAS_CUDA(cudaMemset(P.tc_rounds, 0, ntab));
    std::vector<int2> init(P.tc_tiles, make_int2(INT_MAX, INT_MIN));
    TIDAS_CUDA(cudaMemcpy(P.tc_range, init.data(), P.tc_tiles * 8, cudaMemcpyHostToDevice));
    TIDAS_CUDA(cudaMemset(d_bad, 0, 4));
    long long blocks = ((long long)ntab + 255) / 256;
    das_tc_table_kernel<<<(int)(blocks > 152 * 64 ? 152 * 64 : blocks), 256>>>(
        d, P.tc_tiles_x, P.tc_tiles, P.tc_tab, P.tc_range, d_bad);
    int rc = check_launch("das_tc_table_kernel");
    if (rc) return rc;
    das_tc_round_kernel<<<(P.tc_tiles + 127) / 128, 128>>>(d.n_angles, d.n_elem, P.tc_tiles,
                                                          P.tc_tab, P.tc_range, P.tc_rounds);
    rc = check_launch("das_tc_round_kernel");
    if (rc) return rc;
    int bad = 0;
    TIDAS_CUDA(cudaMemcpy(&bad, d_bad, 4, cudaMemcpyDeviceToHost));
    P.tc_ok = (bad == 0) &&
              dtc::smem_bytes(16, dtc::kMinChunks, d.n_angles, d.n_elem) <= dtc::kSmemMax;
    return TIDAS_OK;
}

int launch_das_tc(const Plan& P, const void* rf, float* img, int nf, cudaStream_t st) {
    using namespace dtc;
    const DasDev& d = P.dev;
    const int A = d.n_angles, NE = d.n_elem, R = A * NE;
    // The widest frame tile (MMA N) up to 64 that the batch fills, preferring
    // one that leaves room for two CTAs per SM; then as many chunks per group
    // ring as the same budget holds.
    int NF = 0;
    size_t budget = kSmemTwoPerSM;
    for (int pass = 0; pass < 2 && !NF; ++pass) {
        budget = pass == 0 ? kSmemTwoPerSM : kSmemMax;
        for (int c = 64; c >= 16 && !NF; c /= 2)
            if ((nf >= c || c == 16) && smem_bytes(c, kMinChunks, A, NE) <= budget) NF = c;
    }
    if (!NF) return set_error(TIDAS_ERR_UNSUPPORTED, "das_tc: tables exceed shared memory");
    int C = kMinChunks;
    while (C < kMaxChunks && smem_bytes(NF, C + 1, A, NE) <= budget) ++C;
    // the plan's staging buffer for the repacked batch (grown on demand)
    const int Sp = packed_len(d.n_samples);
    const int FT = (nf + NF - 1) / NF;
    const size_t need = (size_t)FT * R * Sp * NF * 2;
    // Only the 64-sample blocks that meet the plan's read window (the samples
    // any pixel weights) are packed; the rest of the staging layout is zeroed
    // once, when the buffer comes to this layout, and stays zero.
    void* ws = nullptr;
    bool fresh = false;
    const long long layout = 2 + NF + 256LL * FT;
    if (int rc0 = plan_staging(P, need, &ws, layout, &fresh)) return rc0;
    __half* packed = (__half*)ws;
    if (fresh) TIDAS_CUDA(cudaMemsetAsync(ws, 0, need, st));
    const int rd_lo = P.read_first, rd_hi = P.read_first + P.read_count;
    if (rd_hi > rd_lo) {
        const int sb_first = (rd_lo + kPad) / kPackS, sb_last = (rd_hi - 1 + kPad) / kPackS;
        const int nbw = sb_last - sb_first + 1;
        das_tc_pack_kernel<<<(unsigned)((size_t)FT * R * nbw), 256, 0, st>>>(
            (const __half*)rf, packed, nf, R, d.n_samples, Sp, NF, sb_first, nbw, rd_lo, rd_hi);
        int rc = check_launch("das_tc_pack_kernel");
        if (rc) return rc;
    }
    const size_t smem = smem_bytes(NF, C, A, NE);
    dim3 grid(P.tc_tiles, FT);
    if (d.interp == TIDAS_INTERP_CUBIC) {
        TIDAS_CUDA(cudaFuncSetAttribute(das_tc_kernel<TIDAS_INTERP_CUBIC>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        das_tc_kernel<TIDAS_INTERP_CUBIC><<<grid, kThreads, smem, st>>>(
            packed, d, P.tc_tab, P.tc_range, P.tc_rounds, P.tc_tiles_x, nf, NF, C, img);
    } else {
        TIDAS_CUDA(cudaFuncSetAttribute(das_tc_kernel<TIDAS_INTERP_LINEAR>,
                                        cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem));
        das_tc_kernel<TIDAS_INTERP_LINEAR><<<grid, kThreads, smem, st>>>(
            packed, d, P.tc_tab, P.tc_range, P.tc_rounds, P.tc_tiles_x, nf, NF, C, img);
    }
    return check_launch("das_tc_kernel");
}

}  // namespace tidas
