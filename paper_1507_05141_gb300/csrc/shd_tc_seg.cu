// Stages a1 (project) and a3 (sh2lab) of the mixed-precision path on the
// tcgen05 tensor cores, fed and drained by TMA.
//
// The internal ordinate order is z-class, y-class, x-class (the axis each
// ordinate crosses first), so every class is one contiguous block of the
// discrete-ordinate arrays and shares one sweep layout.  Laboratory-frame
// rows are handled in two groups with a node tiling chosen per group so that
// a tile of 128 nodes is one box of a 5-D tensor map over that layout:
//   group A (z- and y-class): a bw x (128/bw) block of (x, y) at one z,
//   group B (x-class):        a bw x (128/bw) block of (y, z) at one x.
// The group's ordinates are laid out in "slots": each class padded to a
// multiple of the 32-ordinate chunk, so that every chunk is one TMA box
// (class map, 32 ordinates, 128 nodes, one energy group).  Comoving rows of
// moving nodes live node-major ([m][g][k], contiguous in k) in the remap
// scratch and form a third, row-major contraction ("rows" mode) read and
// written through 2-D maps with the 128-byte swizzle.
//
//   a1  D[128 x nb] = A[128 x K] . Bp^T over the item's slots (Bp = [W Y |
//       moment weights], zero at padding slots): group B stores the
//       laboratory moments and the I_lm of nodes at rest, group A adds its
//       part, rows mode stores the I_lm of moving nodes from their comoving
//       intensities.  Warp-specialised: one thread issues TMA boxes into an
//       FP32 staging ring, converter warps split them into BF16 hi / lo in
//       the canonical layout, one thread issues the MMAs into two alternating
//       tensor-memory accumulators, epilogue warps drain them.
//   a3  D[128 x K] = S[128 x NLM] . Y^T: rows mode (k_sh2lab_rows) stores the
//       comoving source S0 of moving nodes node-major for their Lorentz
//       remap; then k_sh2lab_ws, per group, stages eta = chi0 D and chi =
//       chi0 of nodes at rest and the remapped laboratory eta, chi of moving
//       nodes in shared memory and TMA-stores them into the sweep layout.
// FP32 operands are split into BF16 hi + lo and the three products hi.hi +
// hi.lo + lo.hi accumulate in FP32.  Every mbarrier wait is bounded; on
// timeout the kernel raises *err and winds down without hanging.
#include <cuda.h>
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "shd_internal.cuh"
#include "shd_tc.cuh"

namespace shd {

namespace {

constexpr long long kSegWaitLimit = 1LL << 22;  // mbarrier polls before giving up (about a second)
constexpr int kKC = 32;                         // ordinates per chunk
constexpr int kABatch = 8;                      // k_sh2lab_rows: A-build steps whose loads fly together
constexpr int kBox = 128 * kKC;                 // floats per TMA box (16 KB)
constexpr int kNConv = 256;                     // converter threads of a1

__device__ inline void split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
    __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
    hi = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
}

__device__ inline void put1(float *dst, float v, bool acc) { *dst = acc ? *dst + v : v; }
__device__ inline void put4(float *dst, const float *v, bool acc)
{
    float4 o = make_float4(v[0], v[1], v[2], v[3]);
    if (acc) {
        const float4 a = *reinterpret_cast<const float4 *>(dst);
        o.x += a.x; o.y += a.y; o.z += a.z; o.w += a.w;
    }
    *reinterpret_cast<float4 *>(dst) = o;
}

// float4 chunk j of row r of a [rows][32] FP32 tile written with the
// 128-byte swizzle (the tile starts on a 1024-byte boundary)
__device__ inline float4 *swz4(float *tile, int r, int j)
{
    return reinterpret_cast<float4 *>(tile + r * 32 + ((j ^ (r & 7)) << 2));
}

}  // namespace

// Up to four tensor maps per launch: segment mode a1 {class 0, class 1};
// a3 {eta class 0, eta class 1, chi class 0, chi class 1}; rows mode {A}.
struct SegMaps {
    CUtensorMap m[4];
};

// What one launch of the segment / rows kernels covers.
struct SegArgs {
    const int4 *segs;   // segment mode: {plane, a0, b0, 0} (a fastest in the box)
    long long nitem;    // segment mode: segments x G; rows mode: ceil(rows / 128)
    long long nrows;    // rows mode: nmoving x G
    int groupB;         // segment mode: 0 = group A (plane z, a = x, b = y); 1 = B (plane x, a = y, b = z)
    int bw;             // segment mode: box width along a (a power of two, 4..128)
    int nchunk;         // chunks of 32 slots
    int Kp;             // slots = 32 nchunk
    int nb;             // a1: output columns (rows of Bp) of the MMA
    int accumulate;     // a1: add to I_lm / moments instead of storing
    int chi_all;        // a3: chi for every row (else only boxes that hold a moving row)
    int4 chunk[16];     // {map index, first ordinate of the chunk within its class,
                        //  internal index of the class's first ordinate, ordinates in the class}
};

// Index of row r's node within the sweep layout of the class behind map
// `mi` of the tile's group (group A: 0 = z-class (x, y, z), 1 = y-class
// (x, z, y); group B: the x-class (y, z, x)); -1 outside the grid.
__device__ inline long long seg_li(const Prob<float> &P, const SegArgs &S, int4 sd, int r, int mi)
{
    const int a = sd.y + (r & (S.bw - 1)), b = sd.z + r / S.bw;
    if (!S.groupB) {
        if (a >= P.nx || b >= P.ny) return -1;
        return mi == 0 ? ((long long)sd.x * P.ny + b) * P.nx + a : ((long long)b * P.nz + sd.x) * P.nx + a;
    }
    if (a >= P.ny || b >= P.nz) return -1;
    return ((long long)sd.x * P.nz + b) * P.ny + a;
}

// 4-byte asynchronous copy global -> shared; src_size 0 writes a zero and
// reads nothing.
__device__ inline void cp_async4(uint32_t dst, const float *src, uint32_t src_size)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4, %2;\n" ::"r"(dst), "l"(src), "r"(src_size) : "memory");
}
// One arrival on `bar` once every earlier cp.async of this thread has landed
// (the barrier's count already includes it).
__device__ inline void cp_async_arrive(uint64_t *bar)
{
    asm volatile("cp.async.mbarrier.arrive.noinc.shared::cta.b64 [%0];\n" ::"r"(tc::smem_u32(bar)) : "memory");
}
__device__ inline void cp_async_wait_all() { asm volatile("cp.async.wait_all;\n" ::: "memory"); }

// Node of row r of a segment tile; false outside the grid.
__device__ inline bool seg_node(const Prob<float> &P, const SegArgs &S, int4 sd, int r, long long &c)
{
    const int a = sd.y + (r & (S.bw - 1)), b = sd.z + r / S.bw;
    int x, y, z;
    if (!S.groupB) {
        x = a; y = b; z = sd.x;
        if (x >= P.nx || y >= P.ny) return false;
    } else {
        y = a; z = b; x = sd.x;
        if (y >= P.ny || z >= P.nz) return false;
    }
    c = ((long long)z * P.ny + y) * P.nx + x;
    return true;
}

// TMA box coordinates of chunk `ch` of item w.
__device__ inline void box_coords(const SegArgs &S, int ROWS, long long w, int G, int ch, int (&cc)[5])
{
    const int k0 = S.chunk[ch].y;
    if (ROWS) {
        cc[0] = k0;
        cc[1] = (int)(w * 128);
        cc[2] = cc[3] = cc[4] = 0;
        return;
    }
    const long long sg = w / G;
    const int g = (int)(w - sg * G);
    const int4 sd = S.segs[sg];
    // group A: z-class map (x, y, z, g, k), y-class map (x, z, y, g, k);
    // group B: x-class map (y, z, x, g, k)
    const bool yclass = !S.groupB && S.chunk[ch].x == 1;
    cc[0] = sd.y;
    cc[1] = yclass ? sd.x : sd.z;
    cc[2] = yclass ? sd.z : sd.x;
    cc[3] = g;
    cc[4] = k0;
}

// -------------------------------------------------------------------------
// a1.  Warps 0-7 converters, 8-11 epilogue (tensor-memory lane quadrants
// 0-3), 12 TMA producer, 13 MMA issuer.  MAN (planes whose rows are not
// 16-byte multiples, which no tensor map can stride): warps 12 and 14 fill
// the same staging boxes with 4-byte cp.async copies from the sweep layout
// (rows 0-63 and 64-127; zeros outside the grid and past the class's
// ordinates), each lane arriving on the stage's barrier when its copies land.  Shared memory: Bh, Bl [nb][Kp]
// resident; FP32 staging [NSTG][box]; BF16 ring [NR][hi, lo][128][32]
// (canonical); the barriers.  Segment mode: the converters also copy the
// laboratory I of moving rows to nmo, node-major [m][g][k], for the remap.
// -------------------------------------------------------------------------
template <int NSTG, int NR, int ROWS, int MAN>
__global__ void __launch_bounds__(MAN ? 480 : 448, 1)
    k_project_seg(Prob<float> P, const __grid_constant__ SegMaps maps, SegArgs S, const float *__restrict__ Iin,
                  float *__restrict__ Ip, float *__restrict__ mom, float *__restrict__ nmo,
                  const uint16_t *__restrict__ gBh, const uint16_t *__restrict__ gBl, int *err)
{
    static_assert(!(MAN && ROWS), "rows mode always has a tensor map");
    constexpr uint32_t ACC_COLS = 128;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (tc::smem_u32(smem_raw) & 1023) {  // the swizzled staging needs 1024-byte alignment
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    const int Kp = S.Kp, nb = S.nb, nchunk = S.nchunk;
    uint16_t *Bh = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *Bl = Bh + (size_t)nb * Kp;
    float *stg = reinterpret_cast<float *>(Bl + (size_t)nb * Kp);  // [NSTG][kBox]
    uint16_t *ring = reinterpret_cast<uint16_t *>(stg + (size_t)NSTG * kBox);  // [NR][2][128*32]
    uint64_t *sfull = reinterpret_cast<uint64_t *>(ring + (size_t)NR * 2 * 128 * kKC);
    uint64_t *sempty = sfull + NSTG;
    uint64_t *rfull = sempty + NSTG;
    uint64_t *rempty = rfull + NR;
    uint64_t *tfull = rempty + NR;
    uint64_t *tempty = tfull + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = P.G, NLM = P.NLM;
    {
        const uint4 *sh = reinterpret_cast<const uint4 *>(gBh), *sl = reinterpret_cast<const uint4 *>(gBl);
        uint4 *dh = reinterpret_cast<uint4 *>(Bh), *dl = reinterpret_cast<uint4 *>(Bl);
        const int n16 = nb * Kp / 8;
        for (int i = tid; i < n16; i += blockDim.x) {
            dh[i] = sh[i];
            dl[i] = sl[i];
        }
    }
    if (tid == 0) {
        for (int i = 0; i < NSTG; ++i) {
            tc::mbar_init(&sfull[i], MAN ? 64 : 1);
            tc::mbar_init(&sempty[i], kNConv);
        }
        for (int i = 0; i < NR; ++i) {
            tc::mbar_init(&rfull[i], kNConv);
            tc::mbar_init(&rempty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&tfull[i], 1);
            tc::mbar_init(&tempty[i], 128);
        }
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 2 * ACC_COLS);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        for (long long i = 0; i < kSegWaitLimit; ++i) {
            if (tc::mbar_try_wait(bar, parity)) return true;
            if ((i & 255) == 255 && *abort_flag) return false;
        }
        *abort_flag = 1;
        atomicExch(err, 1);
        return false;
    };

    if (warp < 8) {
        // ---------------- converters ----------------
        long long it = 0;
        const int crow = (warp & 3) * 32 + lane;  // the row this thread converts in every chunk
        for (long long w = blockIdx.x; w < S.nitem; w += gridDim.x) {
            // node-major destination of the row when its node moves
            float *nrow = nullptr;
            if (!ROWS && nmo) {
                const long long sg = w / G;
                const int g = (int)(w - sg * G);
                long long c = 0;
                if (seg_node(P, S, S.segs[sg], crow, c)) {
                    const int m = P.midx[c];
                    if (m >= 0) nrow = nmo + ((long long)m * G + g) * P.N;
                }
            }
            for (int ch = 0; ch < nchunk; ++ch, ++it) {
                const int s = (int)(it % NSTG), r = (int)(it % NR);
                if (!wait(&sfull[s], (uint32_t)((it / NSTG) & 1))) goto conv_out;
                if (it >= NR && !wait(&rempty[r], (uint32_t)((it / NR - 1) & 1))) goto conv_out;
                float *Sb = stg + (size_t)s * kBox;
                uint16_t *Ah = ring + (size_t)(2 * r) * 128 * kKC;
                uint16_t *Al = Ah + (size_t)128 * kKC;
                // unit = 32 rows x 8 ordinates (one core-matrix column of
                // four core matrices): lane = row
#pragma unroll
                for (int uu = 0; uu < 2; ++uu) {
                    const int u = warp + 8 * uu;
                    const int rq = u & 3, kb = u >> 2;
                    const int row = rq * 32 + lane;
                    float v[8];
                    if (!ROWS) {
#pragma unroll
                        for (int i = 0; i < 8; ++i) v[i] = Sb[(kb * 8 + i) * 128 + row];
                    } else {
                        const float4 a = *swz4(Sb, row, 2 * kb), b = *swz4(Sb, row, 2 * kb + 1);
                        v[0] = a.x; v[1] = a.y; v[2] = a.z; v[3] = a.w;
                        v[4] = b.x; v[5] = b.y; v[6] = b.z; v[7] = b.w;
                    }
                    uint4 h, l;
                    split2(v[0], v[1], h.x, l.x);
                    split2(v[2], v[3], h.y, l.y);
                    split2(v[4], v[5], h.z, l.z);
                    split2(v[6], v[7], h.w, l.w);
                    const int o = tc::canon_off(row, kb * 8, kKC);
                    *reinterpret_cast<uint4 *>(&Ah[o]) = h;
                    *reinterpret_cast<uint4 *>(&Al[o]) = l;
                    if (!ROWS && nrow) {
                        const int4 ci = S.chunk[ch];
                        const int kl = ci.y + kb * 8;  // within the class
                        float *dst = nrow + ci.z + kl;
                        if (kl + 8 <= ci.w && ((ci.z + kl) & 3) == 0) {
                            reinterpret_cast<float4 *>(dst)[0] = make_float4(v[0], v[1], v[2], v[3]);
                            reinterpret_cast<float4 *>(dst)[1] = make_float4(v[4], v[5], v[6], v[7]);
                        } else {
#pragma unroll
                            for (int i = 0; i < 8; ++i)
                                if (kl + i < ci.w) dst[i] = v[i];
                        }
                    }
                }
                tc::fence_proxy_async();
                tc::mbar_arrive(&sempty[s]);
                tc::mbar_arrive(&rfull[r]);
            }
        }
    conv_out:;
    } else if (MAN && (warp == 12 || warp == 14)) {
        // ---------------- cp.async producers ----------------
        const int r0 = (warp == 12 ? 0 : 64) + lane;  // rows r0 and r0 + 32
        const long long gstride = (long long)G * P.Nc;
        const uint32_t sdst0 = tc::smem_u32(stg) + 4u * (uint32_t)r0;
        long long it = 0;
        for (long long w = blockIdx.x; w < S.nitem; w += gridDim.x) {
            const long long sg = w / G;
            const int g = (int)(w - sg * G);
            const int4 sd = S.segs[sg];
            const long long l00 = seg_li(P, S, sd, r0, 0), l01 = seg_li(P, S, sd, r0 + 32, 0);
            const long long l10 = S.groupB ? -1 : seg_li(P, S, sd, r0, 1);
            const long long l11 = S.groupB ? -1 : seg_li(P, S, sd, r0 + 32, 1);
            for (int ch = 0; ch < nchunk; ++ch, ++it) {
                const int s = (int)(it % NSTG);
                if (it >= NSTG && !wait(&sempty[s], (uint32_t)((it / NSTG - 1) & 1))) goto man_out;
                const int4 ci = S.chunk[ch];
                const long long la = ci.x ? l10 : l00, lb = ci.x ? l11 : l01;
                const float *src = Iin + (long long)(ci.z + ci.y) * gstride + (long long)g * P.Nc;
                const uint32_t d = sdst0 + (uint32_t)s * (kBox * 4);
#pragma unroll 8
                for (int k = 0; k < kKC; ++k, src += gstride) {
                    const bool kin = ci.y + k < ci.w;
                    const bool oa = kin && la >= 0, ob = kin && lb >= 0;
                    cp_async4(d + 512u * k, oa ? src + la : Iin, oa ? 4u : 0u);
                    cp_async4(d + 512u * k + 128u, ob ? src + lb : Iin, ob ? 4u : 0u);
                }
                cp_async_arrive(&sfull[s]);
            }
        }
    man_out:
        cp_async_wait_all();  // no copy may still be landing when the CTA leaves
    } else if (warp == 12) {
        // ---------------- TMA producer ----------------
        if (lane == 0) {
            long long it = 0;
            for (long long w = blockIdx.x; w < S.nitem; w += gridDim.x)
                for (int ch = 0; ch < nchunk; ++ch, ++it) {
                    const int s = (int)(it % NSTG);
                    if (it >= NSTG && !wait(&sempty[s], (uint32_t)((it / NSTG - 1) & 1))) goto prod_out;
                    int cc[5];
                    box_coords(S, ROWS, w, G, ch, cc);
                    tc::mbar_arrive_expect_tx(&sfull[s], kBox * 4);
                    const void *map = &maps.m[S.chunk[ch].x];
                    if (ROWS) tc::tma_load_2d(stg + (size_t)s * kBox, map, cc[0], cc[1], &sfull[s]);
                    else tc::tma_load_5d(stg + (size_t)s * kBox, map, cc[0], cc[1], cc[2], cc[3], cc[4], &sfull[s]);
                }
        prod_out:
            // no copy may still be landing when the CTA leaves
            for (long long i = it > NSTG ? it - NSTG : 0; i < it; ++i)
                tc::mbar_wait(&sfull[i % NSTG], (uint32_t)((i / NSTG) & 1), kSegWaitLimit);
        }
    } else if (warp == 13) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(128, nb);
            const uint32_t a_sbo = (kKC / 8) * 128, b_sbo = (uint32_t)(Kp / 8) * 128;
            const uint32_t bh = tc::smem_u32(Bh), bl = tc::smem_u32(Bl);
            long long it = 0, job = 0;
            bool ok = true;
            for (long long w = blockIdx.x; w < S.nitem && ok; w += gridDim.x, ++job) {
                const int b = (int)(job & 1);
                const long long use = job >> 1;
                if (use > 0 && !wait(&tempty[b], (uint32_t)((use - 1) & 1))) break;
                tc::fence_after_sync();
                const uint32_t d = tmem + (uint32_t)b * ACC_COLS;
                for (int ch = 0; ch < nchunk; ++ch, ++it) {
                    const int r = (int)(it % NR);
                    if (!wait(&rfull[r], (uint32_t)((it / NR) & 1))) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t ah = tc::smem_u32(ring + (size_t)(2 * r) * 128 * kKC);
                    const uint32_t al = ah + 128 * kKC * 2;
#pragma unroll
                    for (int jj = 0; jj < kKC / 16; ++jj) {
                        const uint32_t aoff = jj * 256;
                        const uint32_t boff = (uint32_t)(ch * kKC / 16 + jj) * 256;
                        const uint64_t dah = tc::sdesc(ah + aoff, 128, a_sbo), dal = tc::sdesc(al + aoff, 128, a_sbo);
                        const uint64_t dbh = tc::sdesc(bh + boff, 128, b_sbo), dbl = tc::sdesc(bl + boff, 128, b_sbo);
                        tc::mma_bf16(d, dah, dbh, idesc, (ch > 0 || jj > 0) ? 1u : 0u);
                        tc::mma_bf16(d, dah, dbl, idesc, 1u);
                        tc::mma_bf16(d, dal, dbh, idesc, 1u);
                    }
                    tc::mma_commit(&rempty[r]);
                }
                if (ok) tc::mma_commit(&tfull[b]);
            }
            // no MMA may still be running when the tensor memory is freed
            if (it > 0) tc::mbar_wait(&rempty[(it - 1) % NR], (uint32_t)(((it - 1) / NR) & 1), kSegWaitLimit);
        }
    } else {
        // ---------------- epilogue (warps 8-11) ----------------
        const int quad = warp - 8;
        const int r = quad * 32 + lane;
        const bool acc = S.accumulate != 0;
        const bool sh4 = (NLM & 3) == 0;
        long long job = 0;
        for (long long w = blockIdx.x; w < S.nitem; w += gridDim.x, ++job) {
            // destinations of row r: its I_lm row (when written here) and moments
            float *ip = nullptr, *mp = nullptr;
            if (!ROWS) {
                const long long sg = w / G;
                const int g = (int)(w - sg * G);
                long long c = 0;
                if (seg_node(P, S, S.segs[sg], r, c)) {
                    mp = mom + (c * G + g) * 10;
                    if (P.midx[c] < 0) ip = Ip + (c * G + g) * NLM;
                }
            } else {
                const long long row = w * 128 + r;
                if (row < S.nrows) {
                    const long long m = row / G;
                    ip = Ip + (P.moving[m] * G + (row - m * G)) * NLM;
                }
            }
            // accumulating: the row's previous values, one block of 16 columns
            // ahead of their use (the first block before the accumulator is
            // ready), so that a block's loads are in flight together
            auto load_old = [&](int c0, float (&o)[16]) {
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int col = c0 + 4 * q;
                    if (ip && sh4 && col + 4 <= NLM) {
                        const float4 a4 = *reinterpret_cast<const float4 *>(ip + col);
                        o[4 * q] = a4.x; o[4 * q + 1] = a4.y; o[4 * q + 2] = a4.z; o[4 * q + 3] = a4.w;
                        continue;
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int cc = col + e;
                        o[4 * q + e] = cc < NLM ? (ip ? ip[cc] : 0.f) : (cc < NLM + 10 && mp ? mp[cc - NLM] : 0.f);
                    }
                }
            };
            float oc[16], on[16];
            if (acc) load_old(0, oc);
            const int b = (int)(job & 1);
            if (!wait(&tfull[b], (uint32_t)((job >> 1) & 1))) break;
            tc::fence_after_sync();
            for (int c0 = 0; c0 < nb; c0 += 16) {
                if (acc && c0 + 16 < nb) load_old(c0 + 16, on);
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)b * ACC_COLS + (uint32_t)c0, v);
                if (acc) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) v[i] += oc[i];
                }
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int col = c0 + 4 * q;
                    if (ip && sh4 && col + 4 <= NLM) {
                        put4(ip + col, &v[4 * q], false);
                        continue;
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int cc = col + e;
                        if (cc < NLM) {
                            if (ip) put1(ip + cc, v[4 * q + e], false);
                        } else if (cc < NLM + 10) {
                            if (mp) put1(mp + (cc - NLM), v[4 * q + e], false);
                        }
                    }
                }
                if (acc) {
#pragma unroll
                    for (int i = 0; i < 16; ++i) oc[i] = on[i];
                }
            }
            tc::fence_before_sync();
            tc::mbar_arrive(&tempty[b]);
        }
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * ACC_COLS);
}

// -------------------------------------------------------------------------
// a3.  512 threads, lock-step per item: the rows' S as BF16 hi / lo
// (canonical), the MMAs over the item's slots in column blocks of <= 256,
// then the output chunk by chunk through shared-memory tiles and TMA stores.
// Rows mode: S0 of moving rows (m, g) into node-major rows, two chunks per
// step.  Shared memory: Yh, Yl [Kp][Kq]; A hi / lo [128][Kq]; 4 output tiles
// [box]; per row the S offset; one mbarrier.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(512, 1) k_sh2lab_rows(Prob<float> P, const __grid_constant__ SegMaps maps, SegArgs S,
                                                        const float *__restrict__ Sp, const uint16_t *__restrict__ gYh,
                                                        const uint16_t *__restrict__ gYl, int Kq, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (tc::smem_u32(smem_raw) & 1023) {
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    const int Kp = S.Kp, nchunk = S.nchunk;
    uint16_t *Yh = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *Yl = Yh + (size_t)Kp * Kq;
    uint16_t *Ah = Yl + (size_t)Kp * Kq;
    uint16_t *Al = Ah + (size_t)128 * Kq;
    float *tiles = reinterpret_cast<float *>(Al + (size_t)128 * Kq);  // [4][kBox]
    long long *rsrc = reinterpret_cast<long long *>(tiles + (size_t)4 * kBox);  // [128] S row offset, -1: none
    uint64_t *bar = reinterpret_cast<uint64_t *>(rsrc + 128);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = P.G, NLM = P.NLM;
    {
        const uint4 *sh = reinterpret_cast<const uint4 *>(gYh), *sl = reinterpret_cast<const uint4 *>(gYl);
        uint4 *dh = reinterpret_cast<uint4 *>(Yh), *dl = reinterpret_cast<uint4 *>(Yl);
        const int n16 = Kp * Kq / 8;
        for (int i = tid; i < n16; i += 512) {
            dh[i] = sh[i];
            dl[i] = sl[i];
        }
    }
    if (tid == 0) {
        tc::mbar_init(bar, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t a_sbo = (uint32_t)(Kq / 8) * 128, b_sbo = (uint32_t)(Kq / 8) * 128;
    const int quad = warp & 3, part = warp >> 2;
    uint32_t phase = 0;
    bool pending = false;

    for (long long w = blockIdx.x; w < S.nitem; w += gridDim.x) {
        // the previous item's stores have finished reading the tiles
        if (lane == 0) tc::bulk_wait_read<0>();
        __syncthreads();
        if (tid < 128) {
            long long src = -1;
            const long long row = w * 128 + tid;
            if (row < S.nrows) {
                const long long mm = row / G;
                src = (P.moving[mm] * G + (row - mm * G)) * NLM;
            }
            rsrc[tid] = src;
        }
        __syncthreads();
        // A: the rows' S as BF16 hi / lo, one core matrix per warp step; the
        // loads of kABatch steps are issued together before their stores
        {
            const int j = lane >> 2, kq = lane & 3;
            const int ncm = 16 * (Kq / 8);
            for (int cm0 = warp; cm0 < ncm; cm0 += 16 * kABatch) {
                float v0[kABatch], v1[kABatch];
#pragma unroll
                for (int i = 0; i < kABatch; ++i) {
                    const int cm = cm0 + 16 * i;
                    v0[i] = 0.f;
                    v1[i] = 0.f;
                    if (cm < ncm) {
                        const int rb = cm / (Kq / 8), kb = cm - rb * (Kq / 8);
                        const int row = rb * 8 + j, p = kb * 8 + 2 * kq;
                        const long long src = rsrc[row];
                        if (src >= 0) {
                            if (p < NLM) v0[i] = Sp[src + p];
                            if (p + 1 < NLM) v1[i] = Sp[src + p + 1];
                        }
                    }
                }
#pragma unroll
                for (int i = 0; i < kABatch; ++i) {
                    const int cm = cm0 + 16 * i;
                    if (cm >= ncm) break;
                    const int rb = cm / (Kq / 8), kb = cm - rb * (Kq / 8);
                    const int row = rb * 8 + j, p = kb * 8 + 2 * kq;
                    uint32_t hi, lo;
                    split2(v0[i], v1[i], hi, lo);
                    const int o = tc::canon_off(row, p, Kq);
                    *reinterpret_cast<uint32_t *>(&Ah[o]) = hi;
                    *reinterpret_cast<uint32_t *>(&Al[o]) = lo;
                }
            }
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t ah = tc::smem_u32(Ah), al = tc::smem_u32(Al);
            for (int h = 0; h * 256 < Kp; ++h) {
                const int nh = Kp - 256 * h < 256 ? Kp - 256 * h : 256;
                const uint32_t idesc = tc::idesc_bf16(128, nh);
                const uint32_t yoff = (uint32_t)(256 / 8) * b_sbo * h;
                const uint32_t yh = tc::smem_u32(Yh) + yoff, yl = tc::smem_u32(Yl) + yoff;
                const uint32_t d = tmem + (uint32_t)(256 * h);
                for (int jj = 0; jj < Kq / 16; ++jj) {
                    const uint32_t koff = jj * 256;
                    const uint64_t dah = tc::sdesc(ah + koff, 128, a_sbo), dal = tc::sdesc(al + koff, 128, a_sbo);
                    const uint64_t dbh = tc::sdesc(yh + koff, 128, b_sbo), dbl = tc::sdesc(yl + koff, 128, b_sbo);
                    tc::mma_bf16(d, dah, dbh, idesc, jj > 0 ? 1u : 0u);
                    tc::mma_bf16(d, dah, dbl, idesc, 1u);
                    tc::mma_bf16(d, dal, dbh, idesc, 1u);
                }
            }
            tc::mma_commit(bar);
            pending = true;
            if (!tc::mbar_wait(bar, phase, kSegWaitLimit)) *abort_flag = 1;
            else pending = false;
        }
        __syncthreads();
        if (*abort_flag) goto drain;
        phase ^= 1;
        tc::fence_after_sync();
        {
            const int r = quad * 32 + lane;
            const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
            int cc[5];
            for (int pc = 0; pc * 2 < nchunk; ++pc) {
                float *T0 = tiles + (size_t)((pc & 1) * 2) * kBox;
                // the stores of pair pc - 2 (same tiles) have read them
                if (tid == 0) tc::bulk_wait_read<1>();
                __syncthreads();
                const int chn = 2 * pc + (part >> 1);
                if (chn < nchunk) {
                    float v[16];
                    tc::tmem_ld16(trow + (uint32_t)(chn * kKC + (part & 1) * 16), v);
                    float *T = T0 + (size_t)(part >> 1) * kBox;
#pragma unroll
                    for (int q = 0; q < 4; ++q)
                        *swz4(T, r, (part & 1) * 4 + q) =
                            make_float4(v[4 * q], v[4 * q + 1], v[4 * q + 2], v[4 * q + 3]);
                }
                tc::fence_proxy_async();
                __syncthreads();
                if (tid == 0) {
                    for (int hh = 0; hh < 2 && 2 * pc + hh < nchunk; ++hh) {
                        box_coords(S, 1, w, G, 2 * pc + hh, cc);
                        tc::tma_store_2d(&maps.m[0], cc[0], cc[1], T0 + (size_t)hh * kBox);
                    }
                    tc::bulk_commit();
                }
            }
        }
        tc::fence_before_sync();
        __syncthreads();
    }
    goto done;
drain:
    if (threadIdx.x == 0) {
        atomicExch(err, 1);
        if (pending) tc::mbar_wait(bar, phase, kSegWaitLimit);
    }
done:
    if (lane == 0) tc::bulk_wait_all();
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// -------------------------------------------------------------------------
// a3, segment mode, warp-specialised: the serial phases of an item (building
// A from S, the MMAs) overlap the stores of the previous one.
//   warps 0-7   eta: quadrant warp & 3 of the rows, 16-column half (warp >> 2)
//               of every chunk; wait for a job's accumulator, stage eta in
//               the warp's tile, TMA-store the 32-node x 16-ordinate box
//   warps 8-15  chi: the same boxes of chi (chi0 at rows at rest, the remap's
//               chi at moving rows; runs without a moving row skipped unless
//               every chi is wanted)
//   warps 16-19 A: row (warp - 16) * 32 + lane of the next item: its chi0 and
//               moving index, its S row as BF16 hi / lo (canonical)
//   warp 20     MMA: an item's slots in jobs of <= 256 columns (8 chunks),
//               each into one of two tensor-memory accumulators of 256
//               columns, alternating
// Barriers: metaFull / itemDone per item parity (row tables), aFull / aEmpty
// (the A operand), tFull / tEmpty per accumulator.  MAN (planes whose rows
// are not 16-byte multiples): each epilogue lane writes its own row's 16
// values of a chunk straight into the sweep layout (eta_out, chi_out), one
// coalesced 4-byte store per ordinate, instead of staging a box for TMA.
// -------------------------------------------------------------------------
template <int MAN>
__global__ void __launch_bounds__(672, 1) k_sh2lab_ws(Prob<float> P, const __grid_constant__ SegMaps maps, SegArgs S,
                                                      const float *__restrict__ Sp, const float *__restrict__ etan,
                                                      const float *__restrict__ chin,
                                                      const uint16_t *__restrict__ gYh,
                                                      const uint16_t *__restrict__ gYl, int Kq,
                                                      float *__restrict__ eta_out, float *__restrict__ chi_out,
                                                      int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    if (tc::smem_u32(smem_raw) & 1023) {
        if (threadIdx.x == 0) atomicExch(err, 2);
        return;
    }
    const int Kp = S.Kp, nchunk = S.nchunk;
    uint16_t *Yh = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *Yl = Yh + (size_t)Kp * Kq;
    uint16_t *Ah = Yl + (size_t)Kp * Kq;
    uint16_t *Al = Ah + (size_t)128 * Kq;
    float *tiles = reinterpret_cast<float *>(Al + (size_t)128 * Kq);  // [16 warps][2][16][32]
    float *mchi = tiles + (size_t)16 * 1024;                           // [2][128]
    int *mrow = reinterpret_cast<int *>(mchi + 256);                   // [2][128]
    uint64_t *bars = reinterpret_cast<uint64_t *>(mrow + 256);
    uint64_t *metaFull = bars, *itemDone = bars + 2, *aFull = bars + 4, *aEmpty = bars + 5;
    uint64_t *tFull = bars + 6, *tEmpty = bars + 8;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bars + 10);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int G = P.G, NLM = P.NLM, N = P.N;
    {
        const uint4 *sh = reinterpret_cast<const uint4 *>(gYh), *sl = reinterpret_cast<const uint4 *>(gYl);
        uint4 *dh = reinterpret_cast<uint4 *>(Yh), *dl = reinterpret_cast<uint4 *>(Yl);
        const int n16 = Kp * Kq / 8;
        for (int i = tid; i < n16; i += blockDim.x) {
            dh[i] = sh[i];
            dl[i] = sl[i];
        }
    }
    if (tid == 0) {
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&metaFull[i], 128);
            tc::mbar_init(&itemDone[i], 512);
            tc::mbar_init(&tFull[i], 1);
            tc::mbar_init(&tEmpty[i], 256);
        }
        tc::mbar_init(aFull, 128);
        tc::mbar_init(aEmpty, 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 512);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        for (long long i = 0; i < kSegWaitLimit; ++i) {
            if (tc::mbar_try_wait(bar, parity)) return true;
            if ((i & 255) == 255 && *abort_flag) return false;
        }
        *abort_flag = 1;
        atomicExch(err, 1);
        return false;
    };
    const int njob = (Kp + 255) / 256;  // jobs per item

    if (warp >= 16 && warp < 20) {
        // ---------------- A builders ----------------
        const int r = (warp - 16) * 32 + lane;
        const bool vec = (NLM & 3) == 0;
        // row r of item w: its S offset (-1: none or moving), chi0, moving index
        auto row_of = [&](long long w, long long &src, float &ch, int &m) {
            const long long sg = w / G;
            const int g = (int)(w - sg * G);
            long long c = 0;
            src = -1;
            ch = 0.f;
            m = -1;
            if (seg_node(P, S, S.segs[sg], r, c)) {
                ch = P.chi0[c * G + g];
                m = P.midx[c];
                if (m < 0) src = (c * G + g) * NLM;
            }
        };
        // harmonics [p0, p0 + 32) of the row (16-byte loads when the rows are
        // 16-byte aligned), all in flight together
        auto load_round = [&](long long src, int p0, float (&v)[32]) {
            if (vec) {
#pragma unroll
                for (int q = 0; q < 8; ++q) {
                    const int p = p0 + 4 * q;
                    float4 t = make_float4(0.f, 0.f, 0.f, 0.f);
                    if (src >= 0 && p < NLM) t = *reinterpret_cast<const float4 *>(Sp + src + p);
                    v[4 * q] = t.x; v[4 * q + 1] = t.y; v[4 * q + 2] = t.z; v[4 * q + 3] = t.w;
                }
            } else {
#pragma unroll
                for (int q = 0; q < 32; ++q) v[q] = (src >= 0 && p0 + q < NLM) ? Sp[src + p0 + q] : 0.f;
            }
        };
        auto put_round = [&](int p0, const float (&v)[32]) {
#pragma unroll
            for (int kb = 0; kb < 4; ++kb) {
                if (p0 + kb * 8 >= Kq) break;
                uint4 h, l;
                split2(v[8 * kb], v[8 * kb + 1], h.x, l.x);
                split2(v[8 * kb + 2], v[8 * kb + 3], h.y, l.y);
                split2(v[8 * kb + 4], v[8 * kb + 5], h.z, l.z);
                split2(v[8 * kb + 6], v[8 * kb + 7], h.w, l.w);
                const int o = tc::canon_off(r, p0 + kb * 8, Kq);
                *reinterpret_cast<uint4 *>(&Ah[o]) = h;
                *reinterpret_cast<uint4 *>(&Al[o]) = l;
            }
        };
        // the first round of each item's row is loaded one item ahead (in
        // flight while the A buffer is still in use)
        float v[32];
        long long src = -1;
        float ch = 0.f;
        int m = -1;
        if (blockIdx.x < S.nitem) {
            row_of(blockIdx.x, src, ch, m);
            load_round(src, 0, v);
        }
        long long it = 0;
        for (long long w = blockIdx.x; w < S.nitem; w += gridDim.x, ++it) {
            const int pb = (int)(it & 1);
            if (it >= 2 && !wait(&itemDone[pb], (uint32_t)(((it >> 1) - 1) & 1))) break;
            mchi[pb * 128 + r] = ch;
            mrow[pb * 128 + r] = m;
            tc::mbar_arrive(&metaFull[pb]);
            if (it >= 1 && !wait(aEmpty, (uint32_t)((it - 1) & 1))) break;
            put_round(0, v);
            for (int p0 = 32; p0 < Kq; p0 += 32) {
                load_round(src, p0, v);
                put_round(p0, v);
            }
            tc::fence_proxy_async();
            tc::mbar_arrive(aFull);
            if (w + gridDim.x < S.nitem) {
                row_of(w + gridDim.x, src, ch, m);
                load_round(src, 0, v);
            }
        }
    } else if (warp == 20) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t a_sbo = (uint32_t)(Kq / 8) * 128, b_sbo = (uint32_t)(Kq / 8) * 128;
            const uint32_t ah = tc::smem_u32(Ah), al = tc::smem_u32(Al);
            long long it = 0, j = 0;
            bool ok = true;
            for (long long w = blockIdx.x; w < S.nitem && ok; w += gridDim.x, ++it) {
                if (!wait(aFull, (uint32_t)(it & 1))) break;
                for (int h = 0; h < njob; ++h, ++j) {
                    const int b = (int)(j & 1);
                    if (j >= 2 && !wait(&tEmpty[b], (uint32_t)(((j >> 1) - 1) & 1))) { ok = false; break; }
                    tc::fence_after_sync();
                    const int nh = Kp - 256 * h < 256 ? Kp - 256 * h : 256;
                    const uint32_t idesc = tc::idesc_bf16(128, nh);
                    const uint32_t yoff = (uint32_t)(256 / 8) * b_sbo * h;
                    const uint32_t yh = tc::smem_u32(Yh) + yoff, yl = tc::smem_u32(Yl) + yoff;
                    const uint32_t d = tmem + (uint32_t)(256 * b);
                    for (int jj = 0; jj < Kq / 16; ++jj) {
                        const uint32_t koff = jj * 256;
                        const uint64_t dah = tc::sdesc(ah + koff, 128, a_sbo), dal = tc::sdesc(al + koff, 128, a_sbo);
                        const uint64_t dbh = tc::sdesc(yh + koff, 128, b_sbo), dbl = tc::sdesc(yl + koff, 128, b_sbo);
                        tc::mma_bf16(d, dah, dbh, idesc, jj > 0 ? 1u : 0u);
                        tc::mma_bf16(d, dah, dbl, idesc, 1u);
                        tc::mma_bf16(d, dal, dbh, idesc, 1u);
                    }
                    tc::mma_commit(&tFull[b]);
                }
                if (ok) tc::mma_commit(aEmpty);
            }
            // no MMA may still be running when the tensor memory is freed
            if (it > 0) tc::mbar_wait(aEmpty, (uint32_t)((it - 1) & 1), kSegWaitLimit);
        }
    } else if (warp < 16) {
        // ---------------- epilogue: eta (warps 0-7), chi (8-15) ----------------
        const bool eta_w = warp < 8;
        const int quad = warp & 3, half = (warp >> 2) & 1;
        const int r = quad * 32 + lane;
        const uint32_t trow = tmem + ((uint32_t)(quad * 32) << 16);
        float *W = tiles + (size_t)warp * 1024;  // [2][16][32]
        const float *nsrc = eta_w ? etan : chin;
        const CUtensorMap *mp_base = &maps.m[eta_w ? 0 : 2];
        long long it = 0, j = 0;
        for (long long w = blockIdx.x; w < S.nitem; w += gridDim.x, ++it) {
            const long long sg = w / G;
            const int g = (int)(w - sg * G);
            const int pb = (int)(it & 1);
            const int4 sd = S.segs[sg];
            const int r0 = quad * 32;
            const int as = sd.y + r0 % S.bw, bs = sd.z + r0 / S.bw;
            if (!wait(&metaFull[pb], (uint32_t)((it >> 1) & 1))) break;
            const float chr = mchi[pb * 128 + r];
            const int m = mrow[pb * 128 + r];
            const long long nbase = m >= 0 ? ((long long)m * G + g) * N : 0;
            const bool anym = __any_sync(0xffffffffu, m >= 0);
            // the previous item's stores have read this warp's tiles
            if (!MAN && lane == 0) tc::bulk_wait_read<0>();
            __syncwarp();
            auto store = [&](int cn, const float *src) {
                const int4 ci = S.chunk[cn];
                const int kk = ci.y + 16 * half;
                const bool yc = !S.groupB && ci.x == 1;
                tc::tma_store_5d(mp_base + ci.x, as, yc ? sd.x : bs, yc ? bs : sd.x, g, kk, src);
            };
            // MAN: row r's 16 values of chunk cn, written where they live
            long long li0 = -1, li1 = -1;
            if (MAN) {
                li0 = seg_li(P, S, sd, r, 0);
                li1 = S.groupB ? -1 : seg_li(P, S, sd, r, 1);
            }
            const long long gstride = (long long)G * P.Nc;
            float *const out = eta_w ? eta_out : chi_out;
            auto store_row = [&](int cn, const float (&v)[16]) {
                const int4 ci = S.chunk[cn];
                const long long l = ci.x ? li1 : li0;
                if (l < 0) return;
                const int kl0 = ci.y + 16 * half;
                float *dst = out + (long long)(ci.z + kl0) * gstride + (long long)g * P.Nc + l;
#pragma unroll
                for (int q = 0; q < 16; ++q)
                    if (kl0 + q < ci.w) dst[q * gstride] = v[q];
            };
            // a moving row's 16 values of chunk cn (its own node-major row, 16-byte
            // loads where aligned) into registers, one chunk ahead of their use
            float mv[16];
            auto load_moving = [&](int cn) {
                if (m < 0) return;
                const int4 ci = S.chunk[cn];
                const int kl0 = ci.y + 16 * half;
                const float *src = nsrc + nbase + ci.z + kl0;
                if (kl0 + 16 <= ci.w && ((ci.z + kl0) & 3) == 0) {
#pragma unroll
                    for (int c4 = 0; c4 < 4; ++c4) {
                        const float4 t = reinterpret_cast<const float4 *>(src)[c4];
                        mv[4 * c4] = t.x; mv[4 * c4 + 1] = t.y; mv[4 * c4 + 2] = t.z; mv[4 * c4 + 3] = t.w;
                    }
                } else {
#pragma unroll
                    for (int q = 0; q < 16; ++q) mv[q] = kl0 + q < ci.w ? src[q] : 0.f;
                }
            };
            bool ok = true;
            if (!eta_w && !anym) {
                if (S.chi_all && MAN) {
                    float cv[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) cv[q] = chr;
                    for (int cn = 0; cn < nchunk; ++cn) store_row(cn, cv);
                } else if (S.chi_all) {
                    // every row at rest: one constant chi tile serves every chunk
#pragma unroll
                    for (int q = 0; q < 16; ++q) W[q * 32 + lane] = chr;
                    tc::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        for (int cn = 0; cn < nchunk; ++cn) store(cn, W);
                        tc::bulk_commit();
                    }
                }
            } else {
                if (anym) load_moving(0);
                int jb = -1;  // accumulator of the current job
                for (int cn = 0; cn < nchunk; ++cn) {
                    const int h = cn >> 3;
                    if (eta_w && (cn & 7) == 0) {
                        if (jb >= 0) {
                            tc::fence_before_sync();
                            tc::mbar_arrive(&tEmpty[jb]);
                        }
                        jb = (int)((j + h) & 1);
                        if (!wait(&tFull[jb], (uint32_t)(((j + h) >> 1) & 1))) { ok = false; break; }
                        tc::fence_after_sync();
                    }
                    const int b = cn & 1;
                    if (!MAN && lane == 0) tc::bulk_wait_read<1>();  // the store of chunk cn - 2 has read buffer b
                    __syncwarp();
                    float cur[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) cur[q] = mv[q];
                    if (anym && cn + 1 < nchunk) load_moving(cn + 1);
                    if (MAN) {
                        float o[16];
                        if (eta_w) {
                            float v[16];
                            tc::tmem_ld16(trow + (uint32_t)(256 * jb + (cn & 7) * kKC + 16 * half), v);
#pragma unroll
                            for (int q = 0; q < 16; ++q) o[q] = m < 0 ? chr * v[q] : cur[q];
                        } else {
#pragma unroll
                            for (int q = 0; q < 16; ++q) o[q] = m < 0 ? chr : cur[q];
                        }
                        store_row(cn, o);
                        continue;
                    }
                    float *Wb = W + (size_t)b * 512 + lane;
                    if (eta_w) {
                        float v[16];
                        tc::tmem_ld16(trow + (uint32_t)(256 * jb + (cn & 7) * kKC + 16 * half), v);
#pragma unroll
                        for (int q = 0; q < 16; ++q) Wb[q * 32] = m < 0 ? chr * v[q] : cur[q];
                    } else {
#pragma unroll
                        for (int q = 0; q < 16; ++q) Wb[q * 32] = m < 0 ? chr : cur[q];
                    }
                    tc::fence_proxy_async();
                    __syncwarp();
                    if (lane == 0) {
                        store(cn, W + (size_t)b * 512);
                        tc::bulk_commit();
                    }
                }
                if (eta_w && ok && jb >= 0) {
                    tc::fence_before_sync();
                    tc::mbar_arrive(&tEmpty[jb]);
                }
            }
            if (!ok) break;
            j += njob;
            tc::mbar_arrive(&itemDone[pb]);
        }
        if (!MAN && lane == 0) tc::bulk_wait_all();
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// -------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------
static constexpr size_t kSegSmemLimit = 227 * 1024;

static size_t project_seg_smem(int nb, int Kp, int nstg, int nr)
{
    return (size_t)4 * nb * Kp + (size_t)(nstg + nr) * kBox * 4 + (size_t)(2 * nstg + 2 * nr + 4) * 8 + 8;
}
static size_t sh2lab_seg_smem(int Kp, int Kq)
{
    return (size_t)4 * Kp * Kq + (size_t)4 * 128 * Kq + (size_t)4 * kBox * 4 + 128 * 8 + 8 + 8;
}
static size_t sh2lab_ws_smem(int Kp, int Kq)
{
    return (size_t)4 * Kp * Kq + (size_t)4 * 128 * Kq + (size_t)16 * 1024 * 4 + 2 * 128 * (4 + 4) + 10 * 8 + 8;
}

// staging / ring depths that fit: 0 when nothing does
static int pick_depths(int nb, int Kp, int &nstg, int &nr)
{
    const int opts[4][2] = {{4, 4}, {4, 3}, {4, 2}, {3, 2}};
    for (auto &o : opts)
        if (project_seg_smem(nb, Kp, o[0], o[1]) <= kSegSmemLimit) {
            nstg = o[0];
            nr = o[1];
            return 1;
        }
    return 0;
}

static int nlm16(const shd_ctx *c) { return 16 * ((c->NLM + 15) / 16); }

using EncodeTiled = CUresult (*)(CUtensorMap *, CUtensorMapDataType, cuuint32_t, void *, const cuuint64_t *,
                                 const cuuint64_t *, const cuuint32_t *, const cuuint32_t *, CUtensorMapInterleave,
                                 CUtensorMapSwizzle, CUtensorMapL2promotion, CUtensorMapFloatOOBfill);

static EncodeTiled encoder()
{
    static EncodeTiled fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<EncodeTiled>(p);
    }
    return fn;
}

bool seg_usable(const shd_ctx *c)
{
    if (c->precision != SHD_MIXED || !c->seg_ready || c->NB > 128 || !c->d_tc_Bh || !c->d_tc_Yh || !encoder())
        return false;
    // 16-byte row strides of the node-major maps (the segment tiles of planes
    // whose rows are not 16-byte multiples go through cp.async and plain
    // stores instead of tensor maps)
    if (c->N % 4) return false;
    if (c->tc_Kp > 512 || c->tc_Kp / kKC > 16) return false;
    int a, b;
    for (int grp = 0; grp < 2; ++grp) {
        if (c->tcs_nchunk[grp] == 0) continue;
        if (!c->d_seg[grp] || !c->d_tcs_Bh[grp] || !c->d_tcs_Yh[grp]) return false;
        if (c->tcs_Kp[grp] > 512 || c->tcs_nchunk[grp] > 16) return false;
        if (!pick_depths(c->NB, c->tcs_Kp[grp], a, b)) return false;
        if (sh2lab_ws_smem(c->tcs_Kp[grp], c->tc_Kq) > kSegSmemLimit) return false;
    }
    if (c->nmoving > 0) {
        if (!pick_depths(nlm16(c), c->tc_Kp, a, b)) return false;
        if (sh2lab_seg_smem(c->tc_Kp, c->tc_Kq) > kSegSmemLimit) return false;
    }
    return true;
}

// 5-D map over one class of a discrete-ordinate array: dims (fastest first)
// d0, d1, d2 of the class's sweep layout, then g, then the class's ordinates.
// The box: ba x bb nodes (a fastest) x bk ordinates.
static cudaError_t class_map(const shd_ctx *c, CUtensorMap *m, const float *base, int cls, int ba, int bb, int bk)
{
    const cuuint64_t nx = c->nx, ny = c->ny, nz = c->nz, Nc = (cuuint64_t)c->Nc;
    const int kb = cls == 2 ? 0 : (cls == 1 ? c->nZ : c->nA);
    const int kn = cls == 2 ? c->nZ : (cls == 1 ? c->nA - c->nZ : c->N - c->nA);
    cuuint64_t dims[5], str[4];
    cuuint32_t box[5], es[5] = {1, 1, 1, 1, 1};
    if (cls == 2) {  // (x, y, z)
        dims[0] = nx; dims[1] = ny; dims[2] = nz;
        str[0] = nx * 4; str[1] = nx * ny * 4;
        box[0] = ba; box[1] = bb; box[2] = 1;
    } else if (cls == 1) {  // (x, z, y)
        dims[0] = nx; dims[1] = nz; dims[2] = ny;
        str[0] = nx * 4; str[1] = nx * nz * 4;
        box[0] = ba; box[1] = 1; box[2] = bb;
    } else {  // (y, z, x)
        dims[0] = ny; dims[1] = nz; dims[2] = nx;
        str[0] = ny * 4; str[1] = ny * nz * 4;
        box[0] = ba; box[1] = bb; box[2] = 1;
    }
    dims[3] = (cuuint64_t)c->G;
    dims[4] = (cuuint64_t)kn;
    str[2] = Nc * 4;
    str[3] = (cuuint64_t)c->G * Nc * 4;
    box[3] = 1;
    box[4] = bk;
    void *gaddr = const_cast<float *>(base + (size_t)kb * c->G * Nc);
    CUresult r = encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 5, gaddr, dims, str, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE, CU_TENSOR_MAP_L2_PROMOTION_L2_256B,
                           CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

// 2-D map over node-major rows [R][N], box 32 ordinates x 128 rows, 128-byte swizzle.
static cudaError_t rows_map(const shd_ctx *c, CUtensorMap *m, const float *base)
{
    cuuint64_t dims[2] = {(cuuint64_t)c->N, (cuuint64_t)(c->nmoving * c->G)};
    cuuint64_t str[1] = {(cuuint64_t)c->N * 4};
    cuuint32_t box[2] = {kKC, 128}, es[2] = {1, 1};
    CUresult r = encoder()(m, CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2, const_cast<float *>(base), dims, str, box, es,
                           CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
                           CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS ? cudaSuccess : cudaErrorInvalidValue;
}

static int num_sms_seg(const shd_ctx *ctx)
{
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || n <= 0) n = 148;
    return n;
}

static SegArgs seg_args(const shd_ctx *c, int grp)
{
    SegArgs a{};
    a.segs = (const int4 *)c->d_seg[grp];
    a.nitem = c->nseg[grp] * c->G;
    a.groupB = grp;
    a.bw = c->seg_bw[grp];
    a.nchunk = c->tcs_nchunk[grp];
    a.Kp = c->tcs_Kp[grp];
    for (int i = 0; i < a.nchunk; ++i) {
        const int *t = c->tcs_chunk[grp][i];
        a.chunk[i] = make_int4(t[0], t[1], t[2], t[3]);
    }
    return a;
}

static SegArgs rows_args(const shd_ctx *c)
{
    SegArgs a{};
    a.nrows = c->nmoving * c->G;
    a.nitem = (a.nrows + 127) / 128;
    a.Kp = c->tc_Kp;
    a.nchunk = c->tc_Kp / kKC;
    for (int i = 0; i < a.nchunk; ++i) a.chunk[i] = make_int4(0, i * kKC, 0, c->N);
    return a;
}

// The maps of the classes of group grp (group A {z, y}, group B {x}).  Whole
// tiles (a1 loads): bw x 128/bw nodes x 32 ordinates; quarter tiles (a3
// per-warp stores): 32 consecutive rows of the tile x 16 ordinates.
static cudaError_t group_maps(const shd_ctx *c, int grp, const float *base, CUtensorMap *m0, bool quarter)
{
    const int bw = c->seg_bw[grp];
    const int ba = quarter ? (bw < 32 ? bw : 32) : bw;
    const int bb = quarter ? 32 / ba : 128 / bw;
    const int bk = quarter ? 16 : kKC;
    cudaError_t e;
    if (grp == 0) {
        if (c->nZ > 0 && (e = class_map(c, &m0[0], base, 2, ba, bb, bk)) != cudaSuccess) return e;
        if (c->nA > c->nZ && (e = class_map(c, &m0[1], base, 1, ba, bb, bk)) != cudaSuccess) return e;
        return cudaSuccess;
    }
    return class_map(c, &m0[0], base, 0, ba, bb, bk);
}

// Planes whose rows are not 16-byte multiples: no tensor map can stride
// them, so the segment tiles are loaded by cp.async and stored directly.
bool seg_manual(const shd_ctx *c) { return c->nx % 4 != 0 || c->ny % 4 != 0; }

template <int ROWS, int MAN>
static cudaError_t run_project_seg(const shd_ctx *ctx, const Prob<float> &P, const SegMaps &maps, const SegArgs &a,
                                   const float *I, float *Ip, float *mom, float *nmo, const void *Bh, const void *Bl,
                                   cudaStream_t st)
{
    int nstg = 0, nr = 0;
    if (!pick_depths(a.nb, a.Kp, nstg, nr)) return cudaErrorInvalidConfiguration;
    const size_t sm = project_seg_smem(a.nb, a.Kp, nstg, nr);
    auto kern = nr == 4 ? k_project_seg<4, 4, ROWS, MAN>
                        : (nr == 3 ? k_project_seg<4, 3, ROWS, MAN>
                                   : (nstg == 4 ? k_project_seg<4, 2, ROWS, MAN> : k_project_seg<3, 2, ROWS, MAN>));
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int grid = num_sms_seg(ctx);
    if (a.nitem < grid) grid = (int)a.nitem;
    kern<<<grid, MAN ? 480 : 448, sm, st>>>(P, maps, a, I, Ip, mom, nmo, (const uint16_t *)Bh, (const uint16_t *)Bl,
                                            ctx->d_tc_err);
    note_launch();
    return cudaGetLastError();
}

// a1: the laboratory rows (groups A, B; moving rows also copied node-major
// to nm0), the comoving remap nm0 -> nm1, the comoving rows of moving nodes.
cudaError_t launch_project_seg(const shd_ctx *ctx, const float *I, float *Ip, float *mom, float *nm0, float *nm1,
                               cudaStream_t st)
{
    Prob<float> P = make_prob<float>(ctx);
    bool first = true;
    cudaError_t e;
    // group B (fewer ordinates, short items) stores; group A, whose long items
    // hide the latency of reading back, accumulates
    for (int grp : {1, 0}) {
        if (ctx->tcs_nchunk[grp] == 0 || ctx->nseg[grp] == 0) continue;
        SegArgs a = seg_args(ctx, grp);
        a.nb = ctx->NB;
        a.accumulate = first ? 0 : 1;
        first = false;
        SegMaps maps{};
        float *nmo = ctx->nmoving > 0 ? nm0 : nullptr;
        if (seg_manual(ctx))
            e = run_project_seg<0, 1>(ctx, P, maps, a, I, Ip, mom, nmo, ctx->d_tcs_Bh[grp], ctx->d_tcs_Bl[grp], st);
        else if ((e = group_maps(ctx, grp, I, maps.m, false)) == cudaSuccess)
            e = run_project_seg<0, 0>(ctx, P, maps, a, I, Ip, mom, nmo, ctx->d_tcs_Bh[grp], ctx->d_tcs_Bl[grp], st);
        if (e != cudaSuccess) return e;
    }
    if (ctx->nmoving > 0) {
        if ((e = launch_remap_to_comoving_f(ctx, nm0, nm1, st)) != cudaSuccess) return e;
        SegArgs a = rows_args(ctx);
        a.nb = nlm16(ctx);
        SegMaps maps{};
        if ((e = rows_map(ctx, &maps.m[0], nm1)) != cudaSuccess) return e;
        if ((e = run_project_seg<1, 0>(ctx, P, maps, a, nm1, Ip, mom, nullptr, ctx->d_tc_Bh, ctx->d_tc_Bl, st)) !=
            cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

static cudaError_t run_sh2lab_rows(const shd_ctx *ctx, const Prob<float> &P, const SegMaps &maps, const SegArgs &a,
                                   const float *Sp, const void *Yh, const void *Yl, cudaStream_t st)
{
    const size_t sm = sh2lab_seg_smem(a.Kp, ctx->tc_Kq);
    cudaError_t e = cudaFuncSetAttribute(k_sh2lab_rows, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int grid = num_sms_seg(ctx);
    if (a.nitem < grid) grid = (int)a.nitem;
    k_sh2lab_rows<<<grid, 512, sm, st>>>(P, maps, a, Sp, (const uint16_t *)Yh, (const uint16_t *)Yl, ctx->tc_Kq,
                                         ctx->d_tc_err);
    note_launch();
    return cudaGetLastError();
}

// a3: the comoving S0 of moving nodes (node-major, nm0), their remap to the
// laboratory eta, chi (nm1, nm2), then eta, chi of every node into the sweep
// layout (moving rows taken from nm1, nm2).  Without full_chi, chi is stored
// only for the 32-node runs that hold a moving node; the caller keeps chi0
// in chi_lab at every node at rest (k_chi_rest_fill once per change of chi0
// or of the moving set), so every chi the sweep reads is valid, also in a
// 4-node piece that straddles two rows.
cudaError_t launch_sh2lab_seg(const shd_ctx *ctx, const float *Sp, float *eta, float *chi, float *nm0, float *nm1,
                              float *nm2, cudaStream_t st, bool full_chi)
{
    Prob<float> P = make_prob<float>(ctx);
    cudaError_t e;
    if (ctx->nmoving > 0) {
        SegArgs a = rows_args(ctx);
        SegMaps maps{};
        if ((e = rows_map(ctx, &maps.m[0], nm0)) != cudaSuccess) return e;
        if ((e = run_sh2lab_rows(ctx, P, maps, a, Sp, ctx->d_tc_Yh, ctx->d_tc_Yl, st)) !=
            cudaSuccess)
            return e;
        if ((e = launch_remap_to_lab_f(ctx, nm0, nm1, nm2, st)) != cudaSuccess) return e;
    }
    for (int grp = 0; grp < 2; ++grp) {
        if (ctx->tcs_nchunk[grp] == 0 || ctx->nseg[grp] == 0) continue;
        SegArgs a = seg_args(ctx, grp);
        const bool man = seg_manual(ctx);
        a.chi_all = full_chi ? 1 : 0;
        SegMaps maps{};
        if (!man) {
            if ((e = group_maps(ctx, grp, eta, &maps.m[0], true)) != cudaSuccess) return e;
            if ((e = group_maps(ctx, grp, chi, &maps.m[2], true)) != cudaSuccess) return e;
        }
        auto kern = man ? k_sh2lab_ws<1> : k_sh2lab_ws<0>;
        const size_t sm = sh2lab_ws_smem(a.Kp, ctx->tc_Kq);
        if ((e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) != cudaSuccess)
            return e;
        int grid = num_sms_seg(ctx);
        if (a.nitem < grid) grid = (int)a.nitem;
        kern<<<grid, 672, sm, st>>>(P, maps, a, Sp, nm1, nm2, (const uint16_t *)ctx->d_tcs_Yh[grp],
                                    (const uint16_t *)ctx->d_tcs_Yl[grp], ctx->tc_Kq, eta, chi, ctx->d_tc_err);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    return cudaSuccess;
}

// Self-check of the bounded-wait path: one thread initialises an mbarrier
// that nothing ever arrives on, waits for its first phase with the same
// bounded poll loop the tensor-core kernels use, and raises the context's
// device flag when the wait gives up.  No copy or MMA is in flight, so
// giving up leaves nothing behind.
__global__ void k_wait_selftest(long long polls, int *flag)
{
    __shared__ __align__(8) uint64_t bar;
    if (threadIdx.x != 0) return;
    tc::mbar_init(&bar, 1);
    tc::fence_mbar_init();
    if (!tc::mbar_wait(&bar, 0u, polls)) *flag = 1;
}

cudaError_t launch_wait_selftest(long long polls, int *flag, cudaStream_t st)
{
    k_wait_selftest<<<1, 32, 0, st>>>(polls, flag);
    note_launch();
    return cudaGetLastError();
}

}  // namespace shd
