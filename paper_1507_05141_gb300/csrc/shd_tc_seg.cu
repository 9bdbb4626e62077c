// Stages a1 (project) and a3 (sh2lab) of the mixed-precision path on the
// tcgen05 tensor cores, with every global access a contiguous run.
//
// The internal ordinate order puts the ordinates crossing z or y first
// (group A, [0, nA)) ahead of those crossing x first (group B, [nA, N)).
// Laboratory-frame rows are handled per group with a node tiling chosen so
// that each (ordinate, group) row of a tile is contiguous in that ordinate's
// sweep layout:
//   group A: 128 consecutive nodes of a z-plane in (y, x) order -- one run
//            in the z-layout, runs of nx nodes in the y-layout;
//   group B: 128 consecutive nodes of an x-plane in (z, y) order -- one run
//            in the x-layout.
// A segment item is (segment, energy group g), M = 128 rows.  Comoving rows
// of moving nodes live node-major ([m][g][k], contiguous in k) in the remap
// scratch; they form a third, plain row-major contraction ("rows" mode) over
// 128 consecutive (m, g) rows.
//
//   a1  D[128 x nb] = A[128 x K] . Bp^T   (Bp = [W Y | moment weights] over
//       the item's ordinates): group A stores the laboratory moments and the
//       I_lm of nodes at rest, group B adds its part, rows mode stores the
//       I_lm of moving nodes from their comoving intensities.  Warp-
//       specialised: producers cp.async FP32 rows into a staging ring and
//       convert them to BF16 hi / lo in the canonical layout, one thread
//       issues the MMAs into two alternating tensor-memory accumulators,
//       epilogue warps drain them.
//   a3  D[128 x K] = S[128 x NLM] . Y^T: segment mode writes eta = chi0 D,
//       chi = chi0 of nodes at rest into the sweep layout; rows mode writes
//       the comoving source S0 of moving nodes node-major.
// FP32 operands are split into BF16 hi + lo and the three products hi.hi +
// hi.lo + lo.hi accumulate in FP32.  Every mbarrier wait is bounded; on
// timeout the kernel raises *err and winds down without hanging.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "shd_internal.cuh"
#include "shd_tc.cuh"

namespace shd {

namespace {

constexpr long long kSegWaitLimit = 1LL << 22;  // mbarrier polls before giving up (about a second)
constexpr int kSegKC = 32;                      // ordinates per pipeline chunk
constexpr int kSP = 132;                        // segment staging [k][row] stride (floats)
constexpr int kSR = kSegKC + 8;                 // rows staging [row][k] stride (floats)
constexpr int kNProd = 384;                     // producer threads of a1

__device__ inline void split2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
    __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
    hi = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
}

// Node c of row r of a segment and its offsets in the sweep layouts of the
// group's classes: off2 for z (group A) or x (group B), off1 for y.  False
// beyond the end of the plane.
__device__ inline bool seg_node(const Prob<float> &P, int groupB, int plane, int p0, int r, long long &c,
                                long long &off2, long long &off1)
{
    const int p = p0 + r;
    if (!groupB) {
        const long long PA = (long long)P.nx * P.ny;
        if (p >= PA) return false;
        const int x = p % P.nx, y = p / P.nx, z = plane;
        c = ((long long)z * P.ny + y) * P.nx + x;
        off2 = (long long)z * PA + p;                 // (z, y, x)
        off1 = ((long long)y * P.nz + z) * P.nx + x;  // (y, z, x)
    } else {
        const long long PB = (long long)P.nz * P.ny;
        if (p >= PB) return false;
        const int y = p % P.ny, z = p / P.ny, x = plane;
        c = ((long long)z * P.ny + y) * P.nx + x;
        off2 = (long long)x * PB + p;  // (x, z, y)
        off1 = off2;
    }
    return true;
}

__device__ inline void named_bar(int id, int count)
{
    asm volatile("bar.sync %0, %1;\n" ::"r"(id), "r"(count) : "memory");
}

__device__ inline void cp_async4(float *dst, const float *src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src) : "memory");
}
__device__ inline void cp_async16(float *dst, const float *src)
{
    const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(src) : "memory");
}

// value v into *dst, added to the old value when acc
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

}  // namespace

// What one launch of the segment / rows kernels covers.
struct SegArgs {
    const int4 *segs;  // segment mode: {plane, first in-plane position, 0, 0}
    long long nitem;   // segment mode: segments x G; rows mode: ceil(rows / 128)
    long long nrows;   // rows mode: nmoving x G
    int groupB;        // segment mode: 0 = group A, 1 = group B
    int kbeg, kcnt;    // the ordinates [kbeg, kbeg + kcnt) of the contraction
    int Kp;            // kcnt rounded up to the chunk (a1) or to 16 (a3)
    int nb;            // a1: output columns (rows of Bp) of the MMA
    int accumulate;    // a1: add to I_lm / moments instead of storing
};

// -------------------------------------------------------------------------
// a1.  Warps 0-11 producers, 12-15 epilogue (tensor-memory lane quadrants),
// 16 MMA issuer.  ROWS = 0: segment mode, laboratory I in the sweep layouts;
// ROWS = 1: comoving I0 node-major (row (m, g) = I0 + (m G + g) N).
// Shared memory: Bh, Bl [nb][Kp] resident; ring [NS][hi, lo][128][KC]
// (BF16, canonical); FP32 staging [3] x ([KC][kSP] or [128][kSR]); barriers;
// the classes of the item's ordinates.
// -------------------------------------------------------------------------
template <int NS, int ROWS>
__global__ void __launch_bounds__(544, 1) k_project_seg(Prob<float> P, SegArgs S, const float *__restrict__ A,
                                                        float *__restrict__ Ip, float *__restrict__ mom,
                                                        const uint16_t *__restrict__ gBh,
                                                        const uint16_t *__restrict__ gBl, int *err)
{
    constexpr int KC = kSegKC;
    constexpr uint32_t ACC_COLS = 128;
    constexpr int NCM = 16 * (KC / 8);  // core matrices per chunk
    constexpr int STG = ROWS ? 128 * kSR : KC * kSP;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int Kp = S.Kp, nb = S.nb;
    uint16_t *Bh = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *Bl = Bh + (size_t)nb * Kp;
    uint16_t *ring = Bl + (size_t)nb * Kp;                                   // [NS][2][128*KC]
    float *stg = reinterpret_cast<float *>(ring + (size_t)NS * 2 * 128 * KC);  // [3][STG]
    uint64_t *full = reinterpret_cast<uint64_t *>(stg + (size_t)3 * STG);
    uint64_t *empty = full + NS;
    uint64_t *tfull = empty + NS;
    uint64_t *tempty = tfull + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    volatile int *stop = abort_flag + 1;  // [2] producer decisions, alternating per chunk
    unsigned char *cls = reinterpret_cast<unsigned char *>(tslot + 4);  // [Kp]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = P.N, G = P.G, NLM = P.NLM;
    {
        const uint4 *sh = reinterpret_cast<const uint4 *>(gBh), *sl = reinterpret_cast<const uint4 *>(gBl);
        uint4 *dh = reinterpret_cast<uint4 *>(Bh), *dl = reinterpret_cast<uint4 *>(Bl);
        const int n16 = nb * Kp / 8;
        for (int i = tid; i < n16; i += blockDim.x) {
            dh[i] = sh[i];
            dl[i] = sl[i];
        }
        for (int k = tid; k < Kp; k += blockDim.x) cls[k] = k < S.kcnt ? (unsigned char)P.ord[S.kbeg + k].d : 2;
    }
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            tc::mbar_init(&full[i], kNProd);
            tc::mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            tc::mbar_init(&tfull[i], 1);
            tc::mbar_init(&tempty[i], 128);
        }
        *abort_flag = 0;
        stop[0] = stop[1] = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 2 * ACC_COLS);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;

    const int nchunk = Kp / KC;
    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        for (long long i = 0; i < kSegWaitLimit; ++i) {
            if (tc::mbar_try_wait(bar, parity)) return true;
            if ((i & 255) == 255 && *abort_flag) return false;
        }
        *abort_flag = 1;
        atomicExch(err, 1);
        return false;
    };

    if (warp < 12) {
        // ---------------- producers ----------------
        const int r0 = tid & 127, kslot = tid >> 7;  // segment copies: one row, ordinates kslot + 3i
        const bool vec16 = (N & 3) == 0;
        long long it = 0;
        for (long long w = blockIdx.x; w < S.nitem; w += gridDim.x) {
            // the item's source rows
            long long off2 = 0, off1 = 0, gNc = 0;
            bool valid = false;
            const long long GNc = (long long)G * P.Nc;
            if (!ROWS) {
                const long long sg = w / G;
                const int g = (int)(w - sg * G);
                const int4 sd = S.segs[sg];
                long long c;
                valid = seg_node(P, S.groupB, sd.x, sd.y, r0, c, off2, off1);
                gNc = (long long)g * P.Nc;
            }
            auto copy = [&](int ch, int sb) {
                float *Sb = stg + (size_t)sb * STG;
                if (!ROWS) {
                    for (int kl = kslot; kl < KC; kl += 3) {
                        const int kk = ch * KC + kl;
                        float *dst = &Sb[kl * kSP + r0];
                        if (valid && kk < S.kcnt)
                            cp_async4(dst, A + (long long)(S.kbeg + kk) * GNc + gNc + (cls[kk] == 1 ? off1 : off2));
                        else
                            *dst = 0.f;
                    }
                } else if (vec16) {
                    // 128 rows x KC ordinates as float4: thread -> (row, quad)
                    for (int q = tid; q < 128 * (KC / 4); q += kNProd) {
                        const int r = q / (KC / 4), k4 = (q - r * (KC / 4)) * 4;
                        const long long row = w * 128 + r;
                        const int kk = ch * KC + k4;
                        float *dst = &Sb[r * kSR + k4];
                        if (row < S.nrows && kk < N)
                            cp_async16(dst, A + row * N + kk);
                        else
                            *reinterpret_cast<float4 *>(dst) = make_float4(0.f, 0.f, 0.f, 0.f);
                    }
                } else {
                    for (int q = tid; q < 128 * KC; q += kNProd) {
                        const int r = q / KC, kl = q - r * KC;
                        const long long row = w * 128 + r;
                        const int kk = ch * KC + kl;
                        float *dst = &Sb[r * kSR + kl];
                        if (row < S.nrows && kk < N)
                            cp_async4(dst, A + row * N + kk);
                        else
                            *dst = 0.f;
                    }
                }
                asm volatile("cp.async.commit_group;\n" ::: "memory");
            };
            copy(0, (int)(it % 3));
            if (nchunk > 1) copy(1, (int)((it + 1) % 3));
            for (int ch = 0; ch < nchunk; ++ch, ++it) {
                if (ch + 1 < nchunk) asm volatile("cp.async.wait_group 1;\n" ::: "memory");
                else asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                const int s = (int)(it % NS);
                const long long round = it / NS;
                // one thread waits for ring stage s; the decision reaches every
                // producer through the barrier (slot it & 1 is rewritten only
                // after the next barrier, when everyone has read it)
                if (tid == 0) stop[it & 1] = (round > 0 && !wait(&empty[s], (uint32_t)((round - 1) & 1))) ? 1 : 0;
                named_bar(1, kNProd);  // chunk ch landed everywhere; chunk ch-1 converted; stage s free
                if (stop[it & 1]) {
                    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                    goto prod_out;
                }
                if (ch + 2 < nchunk) copy(ch + 2, (int)((it + 2) % 3));
                const float *Sb = stg + (size_t)(it % 3) * STG;
                uint16_t *Ah = ring + (size_t)(2 * s) * 128 * KC;
                uint16_t *Al = Ah + (size_t)128 * KC;
                // one core matrix (8 rows x 8 ordinates) per warp step:
                // conflict-free staging reads and canonical stores
                const int j = lane >> 2, kq = lane & 3;
                for (int cm = warp; cm < NCM; cm += 12) {
                    const int rb = cm / (KC / 8), kb = cm - rb * (KC / 8);
                    const int row = rb * 8 + j, kl = kb * 8 + 2 * kq;
                    float v0, v1;
                    if (!ROWS) {
                        v0 = Sb[kl * kSP + row];
                        v1 = Sb[(kl + 1) * kSP + row];
                    } else {
                        const float2 t = *reinterpret_cast<const float2 *>(&Sb[row * kSR + kl]);
                        v0 = t.x;
                        v1 = t.y;
                    }
                    uint32_t hi, lo;
                    split2(v0, v1, hi, lo);
                    const int o = tc::canon_off(row, kl, KC);
                    *reinterpret_cast<uint32_t *>(&Ah[o]) = hi;
                    *reinterpret_cast<uint32_t *>(&Al[o]) = lo;
                }
                tc::fence_proxy_async();
                tc::mbar_arrive(&full[s]);
            }
        }
    prod_out:;
    } else if (warp == 16) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(128, nb);
            const uint32_t a_sbo = (KC / 8) * 128, b_sbo = (uint32_t)(Kp / 8) * 128;
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
                    const int s = (int)(it % NS);
                    if (!wait(&full[s], (uint32_t)((it / NS) & 1))) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t ah = tc::smem_u32(ring + (size_t)(2 * s) * 128 * KC);
                    const uint32_t al = ah + 128 * KC * 2;
#pragma unroll
                    for (int jj = 0; jj < KC / 16; ++jj) {
                        const uint32_t aoff = jj * 256;
                        const uint32_t boff = (uint32_t)(ch * KC / 16 + jj) * 256;
                        const uint64_t dah = tc::sdesc(ah + aoff, 128, a_sbo), dal = tc::sdesc(al + aoff, 128, a_sbo);
                        const uint64_t dbh = tc::sdesc(bh + boff, 128, b_sbo), dbl = tc::sdesc(bl + boff, 128, b_sbo);
                        tc::mma_bf16(d, dah, dbh, idesc, (ch > 0 || jj > 0) ? 1u : 0u);
                        tc::mma_bf16(d, dah, dbl, idesc, 1u);
                        tc::mma_bf16(d, dal, dbh, idesc, 1u);
                    }
                    tc::mma_commit(&empty[s]);
                }
                if (ok) tc::mma_commit(&tfull[b]);
            }
        }
    } else if (warp >= 12 && warp < 16) {
        // ---------------- epilogue ----------------
        const int quad = warp - 12;
        const int r = quad * 32 + lane;
        const bool acc = S.accumulate != 0;
        const bool sh4 = (NLM & 3) == 0;
        long long job = 0;
        for (long long w = blockIdx.x; w < S.nitem; w += gridDim.x, ++job) {
            // destination of row r: I_lm row (when written) and moment row
            float *ip = nullptr, *mp = nullptr;
            if (!ROWS) {
                const long long sg = w / G;
                const int g = (int)(w - sg * G);
                const int4 sd = S.segs[sg];
                long long c = 0, o2, o1;
                if (seg_node(P, S.groupB, sd.x, sd.y, r, c, o2, o1)) {
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
            const int b = (int)(job & 1);
            if (!wait(&tfull[b], (uint32_t)((job >> 1) & 1))) break;
            tc::fence_after_sync();
            for (int c0 = 0; c0 < nb; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)b * ACC_COLS + (uint32_t)c0, v);
#pragma unroll
                for (int q = 0; q < 4; ++q) {
                    const int col = c0 + 4 * q;
                    if (ip && sh4 && col + 4 <= NLM) {
                        put4(ip + col, &v[4 * q], acc);
                        continue;
                    }
#pragma unroll
                    for (int e = 0; e < 4; ++e) {
                        const int cc = col + e;
                        if (cc < NLM) {
                            if (ip) put1(ip + cc, v[4 * q + e], acc);
                        } else if (cc < NLM + 10) {
                            if (mp) put1(mp + (cc - NLM), v[4 * q + e], acc);
                        }
                    }
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
// (canonical), the MMAs over the item's ordinates in column blocks of <= 256,
// all 16 warps drain the accumulator (4 per lane quadrant, each a quarter of
// the 16-column blocks).  ROWS = 0: segment mode (rows at rest; eta, chi as
// runs of the sweep layouts); ROWS = 1: moving rows (m, g) -> S0 node-major.
// Shared memory: Yh, Yl [Np][Kq]; A hi / lo [128][Kq]; per row the S offset,
// chi0; one mbarrier; the classes of the item's ordinates.
// -------------------------------------------------------------------------
template <int ROWS>
__global__ void __launch_bounds__(512, 1) k_sh2lab_seg(Prob<float> P, SegArgs S, const float *__restrict__ Sp,
                                                       float *__restrict__ eta, float *__restrict__ chi,
                                                       float *__restrict__ S0, const uint16_t *__restrict__ gYh,
                                                       const uint16_t *__restrict__ gYl, int Kq, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int Np = S.Kp;
    uint16_t *Yh = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *Yl = Yh + (size_t)Np * Kq;
    uint16_t *Ah = Yl + (size_t)Np * Kq;
    uint16_t *Al = Ah + (size_t)128 * Kq;
    long long *rsrc = reinterpret_cast<long long *>(Al + (size_t)128 * Kq);  // [128] S row offset, -1: none
    float *chir = reinterpret_cast<float *>(rsrc + 128);                     // [128]
    uint64_t *bar = reinterpret_cast<uint64_t *>(chir + 128);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    unsigned char *cls = reinterpret_cast<unsigned char *>(tslot + 2);  // [Np]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = P.N, G = P.G, NLM = P.NLM;
    {
        const uint4 *sh = reinterpret_cast<const uint4 *>(gYh), *sl = reinterpret_cast<const uint4 *>(gYl);
        uint4 *dh = reinterpret_cast<uint4 *>(Yh), *dl = reinterpret_cast<uint4 *>(Yl);
        const int n16 = Np * Kq / 8;
        for (int i = tid; i < n16; i += 512) {
            dh[i] = sh[i];
            dl[i] = sl[i];
        }
        for (int k = tid; k < Np; k += 512) cls[k] = k < S.kcnt ? (unsigned char)P.ord[S.kbeg + k].d : 2;
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
    const long long GNc = (long long)G * P.Nc;
    const bool s04 = (N & 3) == 0;
    uint32_t phase = 0;
    bool pending = false;

    for (long long w = blockIdx.x; w < S.nitem; w += gridDim.x) {
        if (tid < 128) {
            long long src = -1;
            float ch = 0.f;
            if (!ROWS) {
                const long long sg = w / G;
                const int g = (int)(w - sg * G);
                const int4 sd = S.segs[sg];
                long long c = 0, o2, o1;
                if (seg_node(P, S.groupB, sd.x, sd.y, tid, c, o2, o1) && P.midx[c] < 0) {
                    src = (c * G + g) * NLM;
                    ch = P.chi0[c * G + g];
                }
            } else {
                const long long row = w * 128 + tid;
                if (row < S.nrows) {
                    const long long m = row / G;
                    src = (P.moving[m] * G + (row - m * G)) * NLM;
                }
            }
            rsrc[tid] = src;
            chir[tid] = ch;
        }
        __syncthreads();
        // A: the rows' S as BF16 hi / lo, one core matrix per warp step
        {
            const int j = lane >> 2, kq = lane & 3;
            for (int cm = warp; cm < 16 * (Kq / 8); cm += 16) {
                const int rb = cm / (Kq / 8), kb = cm - rb * (Kq / 8);
                const int row = rb * 8 + j, p = kb * 8 + 2 * kq;
                const long long src = rsrc[row];
                float v0 = 0.f, v1 = 0.f;
                if (src >= 0) {
                    if (p < NLM) v0 = Sp[src + p];
                    if (p + 1 < NLM) v1 = Sp[src + p + 1];
                }
                uint32_t hi, lo;
                split2(v0, v1, hi, lo);
                const int o = tc::canon_off(row, p, Kq);
                *reinterpret_cast<uint32_t *>(&Ah[o]) = hi;
                *reinterpret_cast<uint32_t *>(&Al[o]) = lo;
            }
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t ah = tc::smem_u32(Ah), al = tc::smem_u32(Al);
            for (int h = 0; h * 256 < Np; ++h) {
                const int nh = Np - 256 * h < 256 ? Np - 256 * h : 256;
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
            const int quad = warp & 3, part = warp >> 2;
            const int r = quad * 32 + lane;
            const bool live = rsrc[r] >= 0;
            const int nblk = Np / 16;
            if (!ROWS) {
                const long long sg = w / G;
                const int g = (int)(w - sg * G);
                const int4 sd = S.segs[sg];
                long long c = 0, off2 = 0, off1 = 0;
                seg_node(P, S.groupB, sd.x, sd.y, r, c, off2, off1);
                const float ch = chir[r];
                const long long gNc = (long long)g * P.Nc;
                for (int blk = part; blk < nblk; blk += 4) {
                    const int c0 = blk * 16;
                    float v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
                    if (!live) continue;
#pragma unroll
                    for (int jj = 0; jj < 16; ++jj) {
                        const int kk = c0 + jj;
                        if (kk < S.kcnt) {
                            const long long a = (long long)(S.kbeg + kk) * GNc + gNc + (cls[kk] == 1 ? off1 : off2);
                            eta[a] = ch * v[jj];
                            chi[a] = ch;
                        }
                    }
                }
            } else {
                float *s0row = S0 + (w * 128 + r) * (long long)N;
                for (int blk = part; blk < nblk; blk += 4) {
                    const int c0 = blk * 16;
                    float v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
                    if (!live) continue;
                    if (s04 && c0 + 16 <= N) {
#pragma unroll
                        for (int q = 0; q < 4; ++q) put4(s0row + c0 + 4 * q, &v[4 * q], false);
                    } else {
#pragma unroll
                        for (int jj = 0; jj < 16; ++jj)
                            if (c0 + jj < N) s0row[c0 + jj] = v[jj];
                    }
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
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// -------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------
static constexpr size_t kSegSmemLimit = 227 * 1024;

static size_t project_seg_smem(int nb, int Kp, int ns, int rows)
{
    const size_t stg = rows ? (size_t)128 * kSR : (size_t)kSegKC * kSP;
    return (size_t)2 * nb * Kp * 2 + (size_t)ns * 2 * 128 * kSegKC * 2 + 3 * stg * 4 + (size_t)(2 * ns + 4) * 8 +
           16 + (size_t)Kp;
}
static size_t sh2lab_seg_smem(int Np, int Kq)
{
    return (size_t)2 * Np * Kq * 2 + (size_t)2 * 128 * Kq * 2 + 128 * 8 + 128 * 4 + 8 + 8 + (size_t)Np;
}

static int pick_ns(int nb, int Kp, int rows)
{
    for (int ns = 4; ns >= 2; --ns)
        if (project_seg_smem(nb, Kp, ns, rows) <= kSegSmemLimit) return ns;
    return 0;
}

// The rows-mode contraction of a1 uses the first nlm16 rows of the full
// projection matrix (the I_lm columns; moments are taken in the laboratory).
static int nlm16(const shd_ctx *c) { return 16 * ((c->NLM + 15) / 16); }

bool seg_usable(const shd_ctx *c)
{
    if (c->precision != SHD_MIXED || c->NB > 128 || !c->d_tc_Bh || !c->d_tc_Yh) return false;
    if (c->tc_Np > 512) return false;
    for (int grp = 0; grp < 2; ++grp) {
        const int cnt = grp ? c->N - c->nA : c->nA;
        if (cnt == 0) continue;
        if (!c->d_seg[grp] || !c->d_tcs_Bh[grp] || !c->d_tcs_Yh[grp]) return false;
        if (c->tcs_Np[grp] > 512) return false;
        if (!pick_ns(c->NB, c->tcs_Kp[grp], 0)) return false;
        if (sh2lab_seg_smem(c->tcs_Np[grp], c->tc_Kq) > kSegSmemLimit) return false;
    }
    if (c->nmoving > 0) {
        if (!pick_ns(nlm16(c), c->tc_Kp, 1)) return false;
        if (sh2lab_seg_smem(c->tc_Np, c->tc_Kq) > kSegSmemLimit) return false;
    }
    return true;
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
    a.kbeg = grp ? c->nA : 0;
    a.kcnt = grp ? c->N - c->nA : c->nA;
    return a;
}

static SegArgs rows_args(const shd_ctx *c)
{
    SegArgs a{};
    a.nrows = c->nmoving * c->G;
    a.nitem = (a.nrows + 127) / 128;
    a.kbeg = 0;
    a.kcnt = c->N;
    return a;
}

template <int ROWS>
static cudaError_t run_project_seg(const shd_ctx *ctx, const Prob<float> &P, SegArgs a, const float *A, float *Ip,
                                   float *mom, const void *Bh, const void *Bl, cudaStream_t st)
{
    const int ns = pick_ns(a.nb, a.Kp, ROWS);
    const size_t sm = project_seg_smem(a.nb, a.Kp, ns, ROWS);
    auto kern = ns == 4 ? k_project_seg<4, ROWS> : (ns == 3 ? k_project_seg<3, ROWS> : k_project_seg<2, ROWS>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int grid = num_sms_seg(ctx);
    if (a.nitem < grid) grid = (int)a.nitem;
    kern<<<grid, 544, sm, st>>>(P, a, A, Ip, mom, (const uint16_t *)Bh, (const uint16_t *)Bl, ctx->d_tc_err);
    return cudaGetLastError();
}

// a1 over the laboratory rows (groups A, B) and the comoving rows of moving
// nodes (I0n node-major).
cudaError_t launch_project_seg(const shd_ctx *ctx, const float *I, float *Ip, float *mom, const float *I0n,
                               cudaStream_t st)
{
    Prob<float> P = make_prob<float>(ctx);
    bool first = true;
    cudaError_t e;
    for (int grp = 0; grp < 2; ++grp) {
        SegArgs a = seg_args(ctx, grp);
        if (a.kcnt == 0 || a.nitem == 0) continue;
        a.Kp = ctx->tcs_Kp[grp];
        a.nb = ctx->NB;
        a.accumulate = first ? 0 : 1;
        first = false;
        if ((e = run_project_seg<0>(ctx, P, a, I, Ip, mom, ctx->d_tcs_Bh[grp], ctx->d_tcs_Bl[grp], st)) != cudaSuccess)
            return e;
    }
    if (ctx->nmoving > 0) {
        SegArgs a = rows_args(ctx);
        a.Kp = ctx->tc_Kp;
        a.nb = nlm16(ctx);
        if ((e = run_project_seg<1>(ctx, P, a, I0n, Ip, mom, ctx->d_tc_Bh, ctx->d_tc_Bl, st)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

template <int ROWS>
static cudaError_t run_sh2lab_seg(const shd_ctx *ctx, const Prob<float> &P, SegArgs a, const float *Sp, float *eta,
                                  float *chi, float *S0n, const void *Yh, const void *Yl, cudaStream_t st)
{
    const size_t sm = sh2lab_seg_smem(a.Kp, ctx->tc_Kq);
    cudaError_t e = cudaFuncSetAttribute(k_sh2lab_seg<ROWS>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int grid = num_sms_seg(ctx);
    if (a.nitem < grid) grid = (int)a.nitem;
    k_sh2lab_seg<ROWS><<<grid, 512, sm, st>>>(P, a, Sp, eta, chi, S0n, (const uint16_t *)Yh, (const uint16_t *)Yl,
                                              ctx->tc_Kq, ctx->d_tc_err);
    return cudaGetLastError();
}

// a3: eta, chi of nodes at rest (groups A, B) and the comoving S0 of moving
// nodes node-major in S0n.
cudaError_t launch_sh2lab_seg(const shd_ctx *ctx, const float *Sp, float *eta, float *chi, float *S0n,
                              cudaStream_t st)
{
    Prob<float> P = make_prob<float>(ctx);
    cudaError_t e;
    for (int grp = 0; grp < 2; ++grp) {
        SegArgs a = seg_args(ctx, grp);
        if (a.kcnt == 0 || a.nitem == 0) continue;
        a.Kp = ctx->tcs_Np[grp];
        if ((e = run_sh2lab_seg<0>(ctx, P, a, Sp, eta, chi, S0n, ctx->d_tcs_Yh[grp], ctx->d_tcs_Yl[grp], st)) !=
            cudaSuccess)
            return e;
    }
    if (ctx->nmoving > 0) {
        SegArgs a = rows_args(ctx);
        a.Kp = ctx->tc_Np;
        if ((e = run_sh2lab_seg<1>(ctx, P, a, Sp, eta, chi, S0n, ctx->d_tc_Yh, ctx->d_tc_Yl, st)) != cudaSuccess)
            return e;
    }
    return cudaSuccess;
}

}  // namespace shd
