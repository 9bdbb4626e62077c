// Stages a1 (project) and a3 (sh2lab) of the mixed-precision path on the
// tcgen05 tensor cores.
//
// Both are contractions over a node brick (8 x 8 nodes in (x, y) at one z)
// and a pair of groups, i.e. M = 128 rows = 2 groups x 64 nodes:
//   a1  D[128 x NB] = A[128 x N] . Bp^T,  A = intensities (laboratory, or
//       comoving for moving nodes), Bp = [W_k Y_p(n_k) | moment weights]
//   a3  D[128 x N]  = S[128 x NLM] . Y^T, then eta = chi0 D, chi = chi0
//       (moving nodes: D to the node-major remap scratch)
// FP32 operands are split into BF16 hi + lo (x = hi + lo to ~16 bits) and
// the three products hi.hi + hi.lo + lo.hi accumulate in FP32 in tensor
// memory; the dropped lo.lo term is below 2^-16 of the result.  The
// right-hand matrix stays resident in shared memory for the whole
// persistent CTA; A chunks are built by the threads in the canonical K-major
// layout and double-buffered against the MMAs with two mbarriers.  Every
// mbarrier wait is bounded: on timeout the kernel raises *err, drains what it
// issued (again bounded), frees its tensor memory and returns.
#include <cuda_bf16.h>
#include <cuda_runtime.h>

#include "shd_internal.cuh"
#include "shd_tc.cuh"

namespace shd {

namespace {

constexpr long long kWaitLimit = 1LL << 22;  // mbarrier polls before giving up (about a second)

__device__ inline int brick_row(int d, int q)
{
    // element q of a run-ordered brick -> row (iy - y0)*8 + (ix - x0); runs
    // follow x in the z- and y-dominant layouts and y in the x-dominant one
    return d == 0 ? ((q & 7) << 3) | (q >> 3) : q;
}

template <class V>
__device__ inline V pick3(int d, V a, V b, V c)
{
    return d == 0 ? a : (d == 1 ? b : c);
}

__device__ inline void split_bf16x2(float a, float b, uint32_t &hi, uint32_t &lo)
{
    __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    __nv_bfloat16 la = __float2bfloat16_rn(a - __bfloat162float(ha));
    __nv_bfloat16 lb = __float2bfloat16_rn(b - __bfloat162float(hb));
    hi = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
}

// one thread waits (bounded), the CTA learns the outcome
__device__ inline bool cta_wait(uint64_t *bar, uint32_t parity, int *abort_flag)
{
    if (threadIdx.x == 0) {
        if (!tc::mbar_wait(bar, parity, kWaitLimit)) *abort_flag = 1;
    }
    __syncthreads();
    return *abort_flag == 0;
}

}  // namespace

// -------------------------------------------------------------------------
// a1 on tensor cores, warp-specialised.  A job is one (brick, group pair,
// pass); every role walks the same job sequence.
//   warps 0-11  producers: cp.async a chunk of KC ordinates for the 128 rows
//               into an FP32 staging area (the next chunk's copies in flight
//               meanwhile), split into BF16 hi / lo, store it in ring stage s
//               in the canonical layout, arrive on full[s]
//   warp  16    MMA issuer (lane 0): wait full[s], 3 x KC/16 MMAs into the
//               job's accumulator (two alternate in tensor memory), commit to
//               empty[s]; after a job's last chunk commit to tfull[b]
//   warps 12-15 epilogue (tensor-memory lane quadrants 0-3): wait tfull[b],
//               read the accumulator, write I_lm / moments, arrive tempty[b]
// Shared memory: Bh, Bl [NB][Kp] resident, the ring [NS][hi, lo][128][KC],
// the FP32 staging [2][KC][128], the barriers, the ordinate layout table.
// -------------------------------------------------------------------------
template <int KC, int NS>
__global__ void __launch_bounds__(544, 1) k_project_tc(Prob<float> P, const float *__restrict__ I,
                                                       const float *__restrict__ I0, float *__restrict__ Ip,
                                                       float *__restrict__ mom, const uint16_t *__restrict__ gBh,
                                                       const uint16_t *__restrict__ gBl, int NB, int Kp, int *err)
{
    constexpr int NPROD = 384;                           // producer threads (warps 0-11)
    constexpr int NPAIR = 128 * KC / 2 / NPROD + 1;      // element pairs a producer covers per chunk (bound)
    constexpr uint32_t ACC_COLS = 128;   // columns per accumulator (NB <= 128)
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint16_t *Bh = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *Bl = Bh + (size_t)NB * Kp;
    uint16_t *ring = Bl + (size_t)NB * Kp;  // [NS][2][128 * KC]
    float *stg = reinterpret_cast<float *>(ring + (size_t)NS * 2 * 128 * KC);  // [2][KC][128]
    uint64_t *full = reinterpret_cast<uint64_t *>(stg + (size_t)2 * KC * 128);
    uint64_t *empty = full + NS;
    uint64_t *tfull = empty + NS;
    uint64_t *tempty = tfull + 2;
    uint32_t *tslot = reinterpret_cast<uint32_t *>(tempty + 2);
    volatile int *abort_flag = reinterpret_cast<volatile int *>(tslot + 1);
    unsigned char *cls = reinterpret_cast<unsigned char *>(tslot + 2);  // [Kp]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = P.N, G = P.G, NLM = P.NLM;
    {
        const uint4 *sh = reinterpret_cast<const uint4 *>(gBh), *sl = reinterpret_cast<const uint4 *>(gBl);
        uint4 *dh = reinterpret_cast<uint4 *>(Bh), *dl = reinterpret_cast<uint4 *>(Bl);
        const int n16 = NB * Kp / 8;
        for (int i = tid; i < n16; i += blockDim.x) {
            dh[i] = sh[i];
            dl[i] = sl[i];
        }
        for (int k = tid; k < Kp; k += blockDim.x) cls[k] = k < N ? (unsigned char)P.ord[k].d : 0;
    }
    if (tid == 0) {
        for (int i = 0; i < NS; ++i) {
            tc::mbar_init(&full[i], NPROD);
            tc::mbar_init(&empty[i], 1);
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

    const int nchunk = Kp / KC;
    const int npair = (G + 1) / 2;
    const long long items = P.ntiles * npair;
    // bounded wait that also gives up as soon as another role has given up
    auto wait = [&](uint64_t *bar, uint32_t parity) -> bool {
        for (long long i = 0; i < kWaitLimit; ++i) {
            if (tc::mbar_try_wait(bar, parity)) return true;
            if ((i & 255) == 255 && *abort_flag) return false;
        }
        *abort_flag = 1;
        atomicExch(err, 1);
        return false;
    };

    if (warp < 12) {
        // ---------------- producers ----------------
        // pair i of a chunk covers ordinates (2 kp, 2 kp + 1), kp = kp0 + 3 i, of
        // row slot q: the slot stays the same because NPROD is a multiple of 128
        const int q = tid & 127, gi = q >> 6, qq = q & 63, kp0 = tid >> 7;
        constexpr int KPS = NPROD / 128;  // pair stride
        long long it = 0;
        for (long long w = blockIdx.x; w < items; w += gridDim.x) {
            const long long tile = w / npair;
            const int pair = (int)(w - tile * npair);
            const TileInfo ti = P.tiles[tile];
            const int passes = (ti.flags & 1) ? 2 : 1;
            const int g = 2 * pair + gi;
            long long off0, off1, off2;
            int row0, row1, row2, m0, m1, m2;
            bool ok0, ok1, ok2;
            {
                auto setup = [&](int d, long long &off, int &row, bool &ok, int &m) {
                    const int rr = brick_row(d, qq);
                    const int ix = ti.x0 + (rr & 7), iy = ti.y0 + (rr >> 3);
                    row = gi * 64 + rr;
                    ok = g < G && ix < P.nx && iy < P.ny;
                    off = ok ? perm_offset(d, ix, iy, ti.z, P.nx, P.ny, P.nz) : 0;
                    m = ok ? P.midx[((long long)ti.z * P.ny + iy) * P.nx + ix] : -1;
                };
                setup(0, off0, row0, ok0, m0);
                setup(1, off1, row1, ok1, m1);
                setup(2, off2, row2, ok2, m2);
            }
            const long long gNc = (long long)(g < G ? g : 0) * P.Nc, GNc = (long long)G * P.Nc;
            for (int pass = 0; pass < passes; ++pass) {
                // element kk of layout d sits at base_d + kk * stride_d: the sweep
                // layout, or in pass 1 the moving node's comoving row; in pass 1
                // the rows of nodes at rest are not needed (zero)
                auto base_of = [&](int m, long long off) -> const float * {
                    return (pass == 1 && m >= 0) ? I0 + ((long long)m * G + g) * N : I + gNc + off;
                };
                const float *base0 = base_of(m0, off0), *base1 = base_of(m1, off1), *base2 = base_of(m2, off2);
                const long long str0 = (pass == 1 && m0 >= 0) ? 1 : GNc;
                const long long str1 = (pass == 1 && m1 >= 0) ? 1 : GNc;
                const long long str2 = (pass == 1 && m2 >= 0) ? 1 : GNc;
                const bool use0 = ok0 && (pass == 0 || m0 >= 0), use1 = ok1 && (pass == 0 || m1 >= 0),
                           use2 = ok2 && (pass == 0 || m2 >= 0);
                // element (kk, q) of a chunk goes to staging [kk][q]: a warp's copies
                // and reads touch consecutive words
                auto copy = [&](int ch, float *S) {
#pragma unroll
                    for (int i = 0; i < NPAIR; ++i) {
#pragma unroll
                        for (int t = 0; t < 2; ++t) {
                            const int kp = kp0 + KPS * i;
                            if (kp >= KC / 2) break;
                            const int kl = 2 * kp + t, kk = ch * KC + kl;
                            float *dst = &S[kl * 128 + q];
                            bool on = false;
                            const float *src = nullptr;
                            if (kk < N) {
                                const int d = cls[kk];
                                if (pick3(d, use0, use1, use2)) {
                                    src = pick3(d, base0, base1, base2) + (long long)kk * pick3(d, str0, str1, str2);
                                    on = true;
                                }
                            }
                            if (on) {
                                const unsigned sa = (unsigned)__cvta_generic_to_shared(dst);
                                asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(sa), "l"(src) : "memory");
                            } else {
                                *dst = 0.f;
                            }
                        }
                    }
                    asm volatile("cp.async.commit_group;\n" ::: "memory");
                };
                copy(0, stg);
                for (int ch = 0; ch < nchunk; ++ch, ++it) {
                    float *S = stg + (size_t)(ch & 1) * KC * 128;
                    if (ch + 1 < nchunk) {
                        copy(ch + 1, stg + (size_t)((ch + 1) & 1) * KC * 128);
                        asm volatile("cp.async.wait_group 1;\n" ::: "memory");
                    } else {
                        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                    }
                    const int s = (int)(it % NS);
                    const long long round = it / NS;
                    if (round > 0 && !wait(&empty[s], (uint32_t)((round - 1) & 1))) {
                        asm volatile("cp.async.wait_group 0;\n" ::: "memory");
                        goto prod_out;
                    }
                    uint16_t *Ah = ring + (size_t)(2 * s) * 128 * KC;
                    uint16_t *Al = Ah + (size_t)128 * KC;
#pragma unroll
                    for (int i = 0; i < NPAIR; ++i) {
                        const int kp = kp0 + KPS * i;
                        if (kp >= KC / 2) break;
                        const int kl = 2 * kp;
                        const int kk = ch * KC + kl;
                        const float v0 = S[kl * 128 + q], v1 = S[(kl + 1) * 128 + q];
                        const int d0 = kk < N ? cls[kk] : 2, d1 = kk + 1 < N ? cls[kk + 1] : 2;
                        const int r0 = kk < N ? pick3(d0, row0, row1, row2) : gi * 64 + qq;
                        const int r1 = kk + 1 < N ? pick3(d1, row0, row1, row2) : gi * 64 + qq;
                        if (r0 == r1) {
                            uint32_t hi, lo;
                            split_bf16x2(v0, v1, hi, lo);
                            const int o = tc::canon_off(r0, kl, KC);
                            *reinterpret_cast<uint32_t *>(&Ah[o]) = hi;
                            *reinterpret_cast<uint32_t *>(&Al[o]) = lo;
                        } else {
                            // the two ordinates use different layouts (different rows for
                            // slot q); each (row, k) is still written once
                            const int rs[2] = {r0, r1};
                            const float vv[2] = {v0, v1};
#pragma unroll
                            for (int t = 0; t < 2; ++t) {
                                __nv_bfloat16 h = __float2bfloat16_rn(vv[t]);
                                __nv_bfloat16 l = __float2bfloat16_rn(vv[t] - __bfloat162float(h));
                                const int o = tc::canon_off(rs[t], kl + t, KC);
                                Ah[o] = __bfloat16_as_ushort(h);
                                Al[o] = __bfloat16_as_ushort(l);
                            }
                        }
                    }
                    tc::fence_proxy_async();
                    tc::mbar_arrive(&full[s]);
                }
            }
        }
    prod_out:;
    } else if (warp == 16) {
        // ---------------- MMA issuer ----------------
        if (lane == 0) {
            const uint32_t idesc = tc::idesc_bf16(128, NB);
            const uint32_t a_sbo = (KC / 8) * 128, b_sbo = (Kp / 8) * 128;
            const uint32_t bh = tc::smem_u32(Bh), bl = tc::smem_u32(Bl);
            long long it = 0, job = 0;
            bool ok = true;
            for (long long w = blockIdx.x; w < items && ok; w += gridDim.x) {
                const TileInfo ti = P.tiles[w / npair];
                const int passes = (ti.flags & 1) ? 2 : 1;
                for (int pass = 0; pass < passes && ok; ++pass, ++job) {
                    const int b = (int)(job & 1);
                    const long long use = job >> 1;
                    if (use > 0 && !wait(&tempty[b], (uint32_t)((use - 1) & 1))) { ok = false; break; }
                    tc::fence_after_sync();
                    const uint32_t d = tmem + (uint32_t)b * ACC_COLS;
                    for (int ch = 0; ch < nchunk; ++ch, ++it) {
                        const int s = (int)(it % NS);
                        if (!wait(&full[s], (uint32_t)((it / NS) & 1))) { ok = false; break; }
                        tc::fence_after_sync();
                        const uint32_t ah = tc::smem_u32(ring + (size_t)(2 * s) * 128 * KC);
                        const uint32_t al = ah + 128 * KC * 2;
#pragma unroll
                        for (int j = 0; j < KC / 16; ++j) {
                            const uint32_t aoff = j * 256;
                            const uint32_t boff = (uint32_t)(ch * KC / 16 + j) * 256;
                            const uint64_t dah = tc::sdesc(ah + aoff, 128, a_sbo), dal = tc::sdesc(al + aoff, 128, a_sbo);
                            const uint64_t dbh = tc::sdesc(bh + boff, 128, b_sbo), dbl = tc::sdesc(bl + boff, 128, b_sbo);
                            tc::mma_bf16(d, dah, dbh, idesc, (ch > 0 || j > 0) ? 1u : 0u);
                            tc::mma_bf16(d, dah, dbl, idesc, 1u);
                            tc::mma_bf16(d, dal, dbh, idesc, 1u);
                        }
                        tc::mma_commit(&empty[s]);
                    }
                    if (ok) tc::mma_commit(&tfull[b]);
                }
            }
        }
    } else if (warp >= 12 && warp < 16) {
        // ---------------- epilogue ----------------
        const int quad = warp - 12;
        const int r = quad * 32 + lane;
        long long job = 0;
        for (long long w = blockIdx.x; w < items; w += gridDim.x) {
            const long long tile = w / npair;
            const int pair = (int)(w - tile * npair);
            const TileInfo ti = P.tiles[tile];
            const int passes = (ti.flags & 1) ? 2 : 1;
            const int egi = r >> 6, rr = r & 63;
            const int eg = 2 * pair + egi;
            const int ix = ti.x0 + (rr & 7), iy = ti.y0 + (rr >> 3);
            const bool valid = eg < G && ix < P.nx && iy < P.ny;
            const long long c = ((long long)ti.z * P.ny + iy) * P.nx + ix;
            const bool moving = valid && P.midx[c] >= 0;
            float *ip = Ip + (c * G + eg) * NLM;
            float *mp = mom + (c * G + eg) * 10;
            for (int pass = 0; pass < passes; ++pass, ++job) {
                const int b = (int)(job & 1);
                if (!wait(&tfull[b], (uint32_t)((job >> 1) & 1))) goto epi_out;
                tc::fence_after_sync();
                const bool write_sh = valid && ((pass == 0 && !moving) || (pass == 1 && moving));
                const bool write_mom = valid && pass == 0;
                for (int c0 = 0; c0 < NB; c0 += 16) {
                    float v[16];
                    tc::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)b * ACC_COLS + (uint32_t)c0, v);
                    if (c0 + 16 <= NLM && (NLM & 3) == 0) {
                        // a full block of harmonics: four 16-byte stores
                        if (write_sh) {
#pragma unroll
                            for (int j = 0; j < 16; j += 4)
                                *reinterpret_cast<float4 *>(&ip[c0 + j]) = make_float4(v[j], v[j + 1], v[j + 2], v[j + 3]);
                        }
                        continue;
                    }
#pragma unroll
                    for (int j = 0; j < 16; ++j) {
                        const int col = c0 + j;
                        if (col < NLM) {
                            if (write_sh) ip[col] = v[j];
                        } else if (col < NLM + 10) {
                            if (write_mom) mp[col - NLM] = v[j];
                        }
                    }
                }
                tc::fence_before_sync();
                tc::mbar_arrive(&tempty[b]);
            }
        }
    epi_out:;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * ACC_COLS);
}

// -------------------------------------------------------------------------
// a3 on tensor cores.  Shared memory: Yh, Yl [Np][Kq] (resident), A hi/lo
// [128][Kq], chi0 and moving flags of the 128 rows, one mbarrier.
// -------------------------------------------------------------------------
__global__ void __launch_bounds__(256, 1) k_sh2lab_tc(Prob<float> P, const float *__restrict__ Sp,
                                                      float *__restrict__ eta, float *__restrict__ chi,
                                                      float *__restrict__ S0, const uint16_t *__restrict__ gYh,
                                                      const uint16_t *__restrict__ gYl, int Np, int Kq, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    uint16_t *Yh = reinterpret_cast<uint16_t *>(smem_raw);
    uint16_t *Yl = Yh + (size_t)Np * Kq;
    uint16_t *Ah = Yl + (size_t)Np * Kq;
    uint16_t *Al = Ah + (size_t)128 * Kq;
    float *chir = reinterpret_cast<float *>(Al + (size_t)128 * Kq);
    int *mrow = reinterpret_cast<int *>(chir + 128);  // moving index of the row, -1 at rest
    uint64_t *bar = reinterpret_cast<uint64_t *>(mrow + 128);
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 1);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    unsigned char *cls = reinterpret_cast<unsigned char *>(abort_flag + 1);  // [Np]

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int N = P.N, G = P.G, NLM = P.NLM;
    {
        const uint4 *sh = reinterpret_cast<const uint4 *>(gYh), *sl = reinterpret_cast<const uint4 *>(gYl);
        uint4 *dh = reinterpret_cast<uint4 *>(Yh), *dl = reinterpret_cast<uint4 *>(Yl);
        const int n16 = Np * Kq / 8;
        for (int i = tid; i < n16; i += 256) {
            dh[i] = sh[i];
            dl[i] = sl[i];
        }
        for (int k = tid; k < Np; k += 256) cls[k] = k < N ? (unsigned char)P.ord[k].d : 0;
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
    const uint32_t a_sbo = (Kq / 8) * 128, b_sbo = (Kq / 8) * 128;
    uint32_t phase = 0;
    bool pending = false;
    const int npair = (G + 1) / 2;
    const long long items = P.ntiles * npair;

    for (long long w = blockIdx.x; w < items; w += gridDim.x) {
        const long long tile = w / npair;
        const int pair = (int)(w - tile * npair);
        const TileInfo ti = P.tiles[tile];
        // rows of S (coalesced along p), split into hi / lo
        for (int e = tid; e < 128 * (Kq / 2); e += 256) {
            const int r = e / (Kq / 2), pp = 2 * (e - r * (Kq / 2));
            const int gi = r >> 6, rr = r & 63;
            const int g = 2 * pair + gi;
            const int ix = ti.x0 + (rr & 7), iy = ti.y0 + (rr >> 3);
            float v0 = 0.f, v1 = 0.f;
            if (g < G && ix < P.nx && iy < P.ny) {
                const long long c = ((long long)ti.z * P.ny + iy) * P.nx + ix;
                const float *row = Sp + (c * G + g) * NLM;
                if (pp < NLM) v0 = row[pp];
                if (pp + 1 < NLM) v1 = row[pp + 1];
            }
            uint32_t hi, lo;
            split_bf16x2(v0, v1, hi, lo);
            const int o = tc::canon_off(r, pp, Kq);
            *reinterpret_cast<uint32_t *>(&Ah[o]) = hi;
            *reinterpret_cast<uint32_t *>(&Al[o]) = lo;
        }
        if (tid < 128) {
            const int r = tid, gi = r >> 6, rr = r & 63, g = 2 * pair + gi;
            const int ix = ti.x0 + (rr & 7), iy = ti.y0 + (rr >> 3);
            float ch = 0.f;
            int m = -1;
            if (g < G && ix < P.nx && iy < P.ny) {
                const long long c = ((long long)ti.z * P.ny + iy) * P.nx + ix;
                ch = P.chi0[c * G + g];
                m = P.midx[c];
            }
            chir[r] = ch;
            mrow[r] = m;
        }
        tc::fence_proxy_async();
        __syncthreads();
        if (tid == 0) {
            tc::fence_after_sync();
            const uint32_t ah = tc::smem_u32(Ah), al = tc::smem_u32(Al);
            for (int h = 0; h * 256 < Np; ++h) {
                const int nh = Np - 256 * h < 256 ? Np - 256 * h : 256;
                const uint32_t idesc = tc::idesc_bf16(128, nh);
                const uint32_t yoff = (uint32_t)(256 * h / 8) * b_sbo;  // 256 rows = 32 core-matrix rows
                const uint32_t yh = tc::smem_u32(Yh) + yoff, yl = tc::smem_u32(Yl) + yoff;
                for (int j = 0; j < Kq / 16; ++j) {
                    const uint32_t koff = j * 256;
                    const uint64_t dah = tc::sdesc(ah + koff, 128, a_sbo), dal = tc::sdesc(al + koff, 128, a_sbo);
                    const uint64_t dbh = tc::sdesc(yh + koff, 128, b_sbo), dbl = tc::sdesc(yl + koff, 128, b_sbo);
                    const uint32_t d = tmem + (uint32_t)(256 * h);
                    tc::mma_bf16(d, dah, dbh, idesc, j > 0 ? 1u : 0u);
                    tc::mma_bf16(d, dah, dbl, idesc, 1u);
                    tc::mma_bf16(d, dal, dbh, idesc, 1u);
                }
            }
            tc::mma_commit(bar);
        }
        pending = true;
        if (!cta_wait(bar, phase, abort_flag)) goto drain;
        phase ^= 1;
        pending = false;
        tc::fence_after_sync();
        {
            // warps w and w+4 share tensor-memory lanes 32*(w%4)..; they split the columns
            const int quad = warp & 3, half = warp >> 2;
            const int r = quad * 32 + lane;
            const int gi = r >> 6, rr = r & 63;
            const int g = 2 * pair + gi;
            const int ix = ti.x0 + (rr & 7), iy = ti.y0 + (rr >> 3);
            const bool valid = g < G && ix < P.nx && iy < P.ny;
            const float ch = chir[r];
            const int mr = mrow[r];
            float *s0row = mr >= 0 ? S0 + ((long long)mr * G + (g < G ? g : 0)) * N : nullptr;
            const long long gNc = (long long)(g < G ? g : 0) * P.Nc;
            const long long off0 = valid ? gNc + perm_offset(0, ix, iy, ti.z, P.nx, P.ny, P.nz) : 0;
            const long long off1 = valid ? gNc + perm_offset(1, ix, iy, ti.z, P.nx, P.ny, P.nz) : 0;
            const long long off2 = valid ? gNc + perm_offset(2, ix, iy, ti.z, P.nx, P.ny, P.nz) : 0;
            const long long GNc = (long long)G * P.Nc;
            const int cbeg = half * (Np / 2), cend = half ? Np : Np / 2;
            for (int c0 = cbeg; c0 < cend; c0 += 16) {
                float v[16];
                tc::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)c0, v);
                if (!valid) continue;
#pragma unroll
                for (int j = 0; j < 16; ++j) {
                    const int k = c0 + j;
                    if (k < N) {
                        if (mr >= 0) {
                            s0row[k] = v[j];  // comoving, node-major
                        } else {
                            const long long a = (long long)k * GNc + pick3((int)cls[k], off0, off1, off2);
                            eta[a] = ch * v[j];
                            chi[a] = ch;
                        }
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
        if (pending) tc::mbar_wait(bar, phase, kWaitLimit);
    }
done:
    tc::fence_before_sync();
    __syncthreads();
    if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

// -------------------------------------------------------------------------
// a2 on tensor cores for kernels that mix groups (Klein-Nishina, Sec. 2.3
// eq:comptoncross): S_lm(c, g) = n_e/chi0 sum_g' K_l[g][g'] I_lm(c, g') + T.
// A tile of TN nodes has, for each l, TN (2l+1) rows (node, m); they are
// taken 128 at a time ("chunks", l by l), each chunk one MMA group
// D[(node, m), g] = sum_g' I(node, g', l, m) K_l[g][g']  (M = 128, K = G'
// padded to Kp, N = G padded to Gp).  Precision: the sums over g' cancel for
// l >= 1 and the spectra span many decades, so each FP32 operand is split
// into three BF16 pieces x = hi + mid + lo (24 significant bits) and the six
// products of order <= 2 (hi.hi, hi.mid, mid.hi, hi.lo, lo.hi, mid.mid)
// accumulate in FP32 in tensor memory: the dropped terms are below 2^-24 of
// each product, as in FP32.  A chunk's operands are built straight from
// I_lm in global memory (every element is read once) while the previous
// chunk's products run (two operand buffers, two accumulators); its
// epilogue finishes S exactly as k_source_sums does (n_e/chi0, emission in
// p = 0, zero where chi0 = 0), stores it and adds the step's FP64 partial
// sums.  Nothing of the tile is staged beyond the operands, so two CTAs
// share an SM.  One thread issues the MMAs; every wait is bounded (on
// timeout: *err raised, what was issued drained, tensor memory freed).
// -------------------------------------------------------------------------
__device__ inline void split3_bf16x2(float a, float b, uint32_t &hi, uint32_t &mid, uint32_t &lo)
{
    const __nv_bfloat16 ha = __float2bfloat16_rn(a), hb = __float2bfloat16_rn(b);
    const float ra = a - __bfloat162float(ha), rb = b - __bfloat162float(hb);
    const __nv_bfloat16 ma = __float2bfloat16_rn(ra), mb = __float2bfloat16_rn(rb);
    const __nv_bfloat16 la = __float2bfloat16_rn(ra - __bfloat162float(ma));
    const __nv_bfloat16 lb = __float2bfloat16_rn(rb - __bfloat162float(mb));
    hi = (uint32_t)__bfloat16_as_ushort(ha) | ((uint32_t)__bfloat16_as_ushort(hb) << 16);
    mid = (uint32_t)__bfloat16_as_ushort(ma) | ((uint32_t)__bfloat16_as_ushort(mb) << 16);
    lo = (uint32_t)__bfloat16_as_ushort(la) | ((uint32_t)__bfloat16_as_ushort(lb) << 16);
}

template <int TN>
__global__ void __launch_bounds__(256, 2) k_source_tc(Prob<float> P, const float *__restrict__ Ip,
                                                      float *__restrict__ Sp, const float *__restrict__ mom,
                                                      const float *__restrict__ Sprev, int have_prev,
                                                      const uint16_t *__restrict__ gK, int Gp, int Kp,
                                                      uint32_t acc_cols, double *partial, int *err)
{
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const int L = P.L, G = P.G, NLM = P.NLM;
    const size_t kblk = (size_t)Gp * Kp;         // elements of one l's operand piece
    const size_t kall = (size_t)(L + 1) * kblk;  // one piece of every l
    const size_t ablk = (size_t)128 * Kp;
    uint16_t *Kop = reinterpret_cast<uint16_t *>(smem_raw);   // [3 pieces][L+1][Gp][Kp]
    uint16_t *Aop = Kop + 3 * kall;                           // [2 buffers][3 pieces][128][Kp]
    float *rat = reinterpret_cast<float *>(Aop + 6 * ablk);   // [TN][G] n_e/chi0 (0 where chi0 = 0)
    float *emt = rat + (size_t)TN * G;                        // [TN][G] sqrt(4 pi) eta0/chi0 (0 there too)
    const size_t tail = ((size_t)(reinterpret_cast<unsigned char *>(emt + (size_t)TN * G) - smem_raw) + 7) & ~(size_t)7;
    uint64_t *bar = reinterpret_cast<uint64_t *>(smem_raw + tail);  // [2] MMA completion
    uint32_t *tslot = reinterpret_cast<uint32_t *>(bar + 2);
    int *abort_flag = reinterpret_cast<int *>(tslot + 1);
    __shared__ double red[4][8];

    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(gK);
        uint4 *dst = reinterpret_cast<uint4 *>(Kop);
        const int n16 = (int)(3 * kall / 8);
        for (int i = tid; i < n16; i += 256) dst[i] = src[i];
    }
    if (tid == 0) {
        tc::mbar_init(&bar[0], 1);
        tc::mbar_init(&bar[1], 1);
        *abort_flag = 0;
        tc::fence_mbar_init();
    }
    if (warp == 0) tc::tmem_alloc(tslot, 2 * acc_cols);
    tc::fence_proxy_async();
    tc::fence_before_sync();
    __syncthreads();
    tc::fence_after_sync();
    const uint32_t tmem = *tslot;
    const uint32_t sbo = (Kp / 8) * 128;
    const uint32_t idesc = tc::idesc_bf16(128, Gp);
    uint32_t mphase[2] = {0, 0};
    bool mpend[2] = {false, false};
    double e_sum = 0, ph_sum = 0, num = 0, den = 0;
    const long long ntiles = (P.Nc + TN - 1) / TN;
    const size_t nstride = (size_t)G * NLM;  // floats per node in I_lm / S_lm

    // chunk q of l: rows q*128 + r, r < 128, of the tile's (node, m) rows
    // (node = row / (2l+1), p = l^2 + row % (2l+1)); nch(l) chunks per l
    auto nch = [&](int l, int nn) { return (nn * (2 * l + 1) + 127) / 128; };
    // operands of (l, q) into buffer b, straight from I_lm: a warp's threads
    // take consecutive rows (consecutive p within a node)
    auto build = [&](long long c0, int nn, int l, int q, int b) {
        const int nm = 2 * l + 1, rows = nn * nm, p0 = l * l, r0 = q * 128;
        uint16_t *Ah = Aop + (size_t)(3 * b) * ablk, *Am = Ah + ablk, *Al = Am + ablk;
#pragma unroll 4
        for (int e = tid; e < 128 * (Kp / 2); e += 256) {
            const int r = e & 127, kk = 2 * (e >> 7);
            float v0 = 0.f, v1 = 0.f;
            const int row = r0 + r;
            if (row < rows) {
                const int node = row / nm, p = p0 + (row - node * nm);
                const float *bp = Ip + (size_t)(c0 + node) * nstride + p;
                if (kk < G) v0 = __ldg(bp + (size_t)kk * NLM);
                if (kk + 1 < G) v1 = __ldg(bp + (size_t)(kk + 1) * NLM);
            }
            uint32_t hi, mid, lo;
            split3_bf16x2(v0, v1, hi, mid, lo);
            const int o = tc::canon_off(r, kk, Kp);
            *reinterpret_cast<uint32_t *>(&Ah[o]) = hi;
            *reinterpret_cast<uint32_t *>(&Am[o]) = mid;
            *reinterpret_cast<uint32_t *>(&Al[o]) = lo;
        }
    };
    // the six products of buffer b's operands with K_l into accumulator b
    auto issue = [&](int l, int b) {
        tc::fence_after_sync();
        const uint32_t a0 = tc::smem_u32(Aop + (size_t)(3 * b) * ablk);
        const uint32_t ap[3] = {a0, a0 + (uint32_t)(ablk * 2), a0 + (uint32_t)(ablk * 4)};
        const uint32_t k0 = tc::smem_u32(Kop + (size_t)l * kblk);
        const uint32_t kp[3] = {k0, k0 + (uint32_t)(kall * 2), k0 + (uint32_t)(kall * 4)};
        const int pa[6] = {0, 0, 1, 0, 2, 1}, pb[6] = {0, 1, 0, 2, 0, 1};
        const uint32_t d = tmem + (uint32_t)b * acc_cols;
        for (int j = 0; j < Kp / 16; ++j) {
            const uint32_t koff = j * 256;
#pragma unroll
            for (int qq = 0; qq < 6; ++qq) {
                const uint64_t da = tc::sdesc(ap[pa[qq]] + koff, 128, sbo), db = tc::sdesc(kp[pb[qq]] + koff, 128, sbo);
                tc::mma_bf16(d, da, db, idesc, (j > 0 || qq > 0) ? 1u : 0u);
            }
        }
        tc::mma_commit(&bar[b]);
    };
    // accumulator b of (l, q): S = n_e/chi0 D + emission (p = 0) straight to
    // S_lm, with the partial sums of |S|^2 and |S - S_prev|^2
    auto epilogue = [&](long long c0, int nn, int l, int q, int b) {
        const int nm = 2 * l + 1, rows = nn * nm, p0 = l * l;
        // warps w and w+4 share tensor-memory lanes 32 (w % 4) ..; they split the columns
        const int quad = warp & 3, half = warp >> 2;
        const int r = quad * 32 + lane, row = q * 128 + r;
        const bool valid = row < rows;
        const int node = valid ? row / nm : 0, p = p0 + (valid ? row - node * nm : 0);
        const size_t obase = (size_t)(c0 + node) * nstride + p;
        const int cb = half * (Gp / 2), ce = half ? Gp : Gp / 2;
        // this row's part of |S|^2 and |S - S_prev|^2 in FP32, added to the
        // FP64 totals once (an FP64 operation per output would occupy the
        // narrow FP64 pipe)
        float dn = 0.f, nmr = 0.f;
        for (int cc = cb; cc < ce; cc += 16) {
            float v[16];
            tc::tmem_ld16(tmem + ((uint32_t)(quad * 32) << 16) + (uint32_t)b * acc_cols + (uint32_t)cc, v);
            if (!valid) continue;
#pragma unroll
            for (int j = 0; j < 16; ++j) {
                const int g = cc + j;
                if (g >= G) break;
                float sv = rat[node * G + g] * v[j];
                if (p == 0) sv += emt[node * G + g];
                const size_t o = obase + (size_t)g * NLM;
                Sp[o] = sv;
                dn += sv * sv;
                if (have_prev) {
                    const float dd = sv - Sprev[o];
                    nmr += dd * dd;
                }
            }
        }
        den += (double)dn;
        num += (double)nmr;
    };

    for (long long w = blockIdx.x; w < ntiles; w += gridDim.x) {
        const long long c0 = w * TN;
        const int nn = (int)(P.Nc - c0 < TN ? P.Nc - c0 : TN);
        for (int i = tid; i < nn * G; i += 256) {
            const long long c = c0 + i / G;
            const float chi = P.chi0[c * G + (i % G)];
            rat[i] = chi > 0.f ? P.ne[c] / chi : 0.f;
            emt[i] = chi > 0.f ? 3.5449077018110320546f * P.emis0[c * G + (i % G)] / chi : 0.f;  // sqrt(4 pi)
            const int g = i % G;
            const double J = (double)mom[(c * G + g) * 10];
            const double de = P.edges[g + 1] - P.edges[g];
            e_sum += 4.0 * kPi * J * de;
            ph_sum += 4.0 * kPi * J * de / P.centre[g];
        }
        // the tile's chunks in order (l, q), software-pipelined: chunk i+1's
        // operands are built while chunk i's products run
        int l = 0, q = 0, b = 0;
        build(c0, nn, 0, 0, 0);
        tc::fence_proxy_async();
        __syncthreads();  // also makes rat / emt visible
        if (tid == 0) issue(0, 0);
        mpend[0] = true;
        while (true) {
            // next chunk after (l, q)
            int ln = l, qn = q + 1;
            if (qn >= nch(l, nn)) { ln = l + 1; qn = 0; }
            const bool more = ln <= L;
            if (more) build(c0, nn, ln, qn, b ^ 1);  // accumulator b ^ 1 was drained by the previous epilogue
            tc::fence_proxy_async();
            tc::fence_before_sync();
            __syncthreads();
            if (more) {
                if (tid == 0) issue(ln, b ^ 1);
                mpend[b ^ 1] = true;
            }
            if (!cta_wait(&bar[b], mphase[b], abort_flag)) goto drain;
            mphase[b] ^= 1;
            mpend[b] = false;
            tc::fence_after_sync();
            epilogue(c0, nn, l, q, b);
            tc::fence_before_sync();
            if (!more) break;
            l = ln;
            q = qn;
            b ^= 1;
        }
        __syncthreads();  // rat / emt are rewritten by the next tile
    }
    goto done;
drain:
    if (threadIdx.x == 0) {
        atomicExch(err, 1);
        for (int bb = 0; bb < 2; ++bb)
            if (mpend[bb]) tc::mbar_wait(&bar[bb], mphase[bb], kWaitLimit);
    }
done:
    // fixed-order reduction of the partial sums: lanes, then the 8 warps
    for (int o = 16; o > 0; o >>= 1) {
        e_sum += __shfl_down_sync(0xffffffffu, e_sum, o);
        ph_sum += __shfl_down_sync(0xffffffffu, ph_sum, o);
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if (lane == 0) {
        red[0][warp] = e_sum;
        red[1][warp] = ph_sum;
        red[2][warp] = num;
        red[3][warp] = den;
    }
    tc::fence_before_sync();
    __syncthreads();
    if (tid < 4) {
        double acc = 0;
        for (int qq = 0; qq < 8; ++qq) acc += red[tid][qq];
        partial[blockIdx.x * 4 + tid] = acc;
    }
    if (warp == 0) tc::tmem_dealloc(tmem, 2 * acc_cols);
}

// Three BF16 pieces hi, mid, lo of K_l[g][g'] (FP32 [L+1][G][G]) in the
// canonical K-major layout of the source MMA: [piece][l][Gp][Kp], row g,
// column g', zero padded.
__global__ void k_source_tc_operands(const float *__restrict__ K, int L, int G, int Gp, int Kp, uint16_t *out)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long all = (long long)(L + 1) * Gp * Kp;
    if (i >= all) return;
    const int l = (int)(i / ((long long)Gp * Kp));
    const int rem = (int)(i - (long long)l * Gp * Kp);
    const int g = rem / Kp, gp = rem - g * Kp;
    const float v = (g < G && gp < G) ? K[((size_t)l * G + g) * G + gp] : 0.f;
    const __nv_bfloat16 h = __float2bfloat16_rn(v);
    const float r = v - __bfloat162float(h);
    const __nv_bfloat16 m = __float2bfloat16_rn(r);
    const __nv_bfloat16 lo = __float2bfloat16_rn(r - __bfloat162float(m));
    const size_t o = (size_t)l * Gp * Kp + tc::canon_off(g, gp, Kp);
    out[o] = __bfloat16_as_ushort(h);
    out[all + o] = __bfloat16_as_ushort(m);
    out[2 * all + o] = __bfloat16_as_ushort(lo);
}

// -------------------------------------------------------------------------
// host side
// -------------------------------------------------------------------------
static constexpr int kProjKC = 32;

static size_t project_tc_smem_ns(const shd_ctx *c, int ns)
{
    return (size_t)2 * c->NB * c->tc_Kp * 2 + (size_t)ns * 2 * 128 * kProjKC * 2 + (size_t)2 * kProjKC * 128 * 4 +
           (2 * ns + 4) * 8 + 16 + (size_t)c->tc_Kp;
}
size_t project_tc_smem_bytes(const shd_ctx *c) { return project_tc_smem_ns(c, 2); }
size_t sh2lab_tc_smem_bytes(const shd_ctx *c)
{
    return (size_t)2 * c->tc_Np * c->tc_Kq * 2 + (size_t)2 * 128 * c->tc_Kq * 2 + 128 * 4 + 128 * 4 + 64 +
           (size_t)c->tc_Np;
}

bool tc_usable(const shd_ctx *c)
{
    if (c->precision != SHD_MIXED || !c->d_tc_Bh || !c->d_tc_Yh) return false;
    if (c->NB > 128 || c->tc_Np > 512) return false;
    return project_tc_smem_bytes(c) <= 227 * 1024 && sh2lab_tc_smem_bytes(c) <= 227 * 1024;
}

static int num_sms_tc(const shd_ctx *ctx)
{
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || n <= 0) n = 148;
    return n;
}

cudaError_t launch_project_tc(const shd_ctx *ctx, const float *I, float *Ip, float *mom, const float *I0n,
                              cudaStream_t st)
{
    Prob<float> P = make_prob<float>(ctx);
    const bool three = project_tc_smem_ns(ctx, 3) <= 227 * 1024;
    size_t sm = project_tc_smem_ns(ctx, three ? 3 : 2);
    auto kern = three ? k_project_tc<kProjKC, 3> : k_project_tc<kProjKC, 2>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    long long items = ctx->ntiles * ((ctx->G + 1) / 2);
    int grid = num_sms_tc(ctx);
    if (items < grid) grid = (int)items;
    kern<<<grid, 544, sm, st>>>(P, I, I0n, Ip, mom, (const uint16_t *)ctx->d_tc_Bh, (const uint16_t *)ctx->d_tc_Bl,
                                ctx->NB, ctx->tc_Kp, ctx->d_tc_err);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_sh2lab_tc(const shd_ctx *ctx, const float *Sp, float *eta, float *chi, float *S0n, cudaStream_t st)
{
    Prob<float> P = make_prob<float>(ctx);
    size_t sm = sh2lab_tc_smem_bytes(ctx);
    cudaError_t e = cudaFuncSetAttribute(k_sh2lab_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    long long items = ctx->ntiles * ((ctx->G + 1) / 2);
    int grid = num_sms_tc(ctx);
    if (items < grid) grid = (int)items;
    k_sh2lab_tc<<<grid, 256, sm, st>>>(P, Sp, eta, chi, S0n, (const uint16_t *)ctx->d_tc_Yh,
                                      (const uint16_t *)ctx->d_tc_Yl, ctx->tc_Np, ctx->tc_Kq, ctx->d_tc_err);
    note_launch();
    return cudaGetLastError();
}

// ---- the tensor-core source (a2) ------------------------------------------

static int round16(int x) { return (x + 15) / 16 * 16; }

// Nodes per tile of k_source_tc and its shared memory: operands of every l
// (three pieces), two operand buffers, the tile's n_e/chi0 and emission; 0
// when that exceeds what two CTAs per SM can share (113 KB each).
static int source_tc_tn(const shd_ctx *c, size_t *smem)
{
    const int Gp = round16(c->G), Kp = round16(c->G);
    const int tn = 64;
    const size_t sm = (size_t)3 * (c->L + 1) * Gp * Kp * 2 + (size_t)6 * 128 * Kp * 2 + (size_t)2 * tn * c->G * 4 +
                      8 + 2 * 8 + 16;
    if (sm > 113 * 1024) return 0;  // two CTAs and their 1 KB reservations fill the SM's 228 KB
    if (smem) *smem = sm;
    return tn;
}

bool source_tc_usable(const shd_ctx *c)
{
    return c->precision == SHD_MIXED && !c->k_diagonal && c->scat_kind != SHD_SCAT_KN_THERMAL && c->G <= 256 &&
           c->d_tcK && source_tc_tn(c, nullptr) > 0;
}

cudaError_t launch_source_tc_operands(shd_ctx *c, cudaStream_t st)
{
    const int Gp = round16(c->G), Kp = round16(c->G);
    const size_t n = (size_t)(c->L + 1) * Gp * Kp;
    k_source_tc_operands<<<(unsigned)((n + 255) / 256), 256, 0, st>>>((const float *)c->d_K, c->L, c->G, Gp, Kp,
                                                                     (uint16_t *)c->d_tcK);
    note_launch();
    return cudaGetLastError();
}

size_t source_tc_operand_bytes(const shd_ctx *c)
{
    return (size_t)3 * (c->L + 1) * round16(c->G) * round16(c->G) * sizeof(uint16_t);
}

cudaError_t launch_source_sums_tc(shd_ctx *c, const float *Ip, float *Sp, const float *mom, const float *Sprev,
                                  bool have_prev, int *grid_used, cudaStream_t st)
{
    Prob<float> P = make_prob<float>(c);
    size_t sm = 0;
    const int tn = source_tc_tn(c, &sm);
    const int Gp = round16(c->G), Kp = round16(c->G);
    uint32_t cols = 32;
    while ((int)cols < Gp) cols <<= 1;
    const uint16_t *Kop = (const uint16_t *)c->d_tcK;
    // persistent: two CTAs per SM (no more than there are tiles); every CTA
    // loads the K operands once
    const long long ntiles = (c->Nc + tn - 1) / tn;
    long long nbl = 2LL * num_sms_tc(c);
    if (nbl > ntiles) nbl = ntiles;
    if (nbl > c->n_partial) nbl = c->n_partial;
    const int nb = (int)nbl;
    if (grid_used) *grid_used = nb;
    cudaError_t e;
#define SHD_SRC_TC(T)                                                                                         \
    case T:                                                                                                   \
        if ((e = cudaFuncSetAttribute(k_source_tc<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm)) !=  \
            cudaSuccess)                                                                                      \
            return e;                                                                                         \
        /* all of the SM's unified memory as shared memory: two CTAs fit */                                   \
        if ((e = cudaFuncSetAttribute(k_source_tc<T>, cudaFuncAttributePreferredSharedMemoryCarveout, 100)) !=   \
            cudaSuccess)                                                                                      \
            return e;                                                                                         \
        k_source_tc<T><<<nb, 256, sm, st>>>(P, Ip, Sp, mom, Sprev, have_prev ? 1 : 0, Kop, Gp, Kp, cols,       \
                                            c->d_partial, c->d_tc_err);                                       \
        break;
    switch (tn) {
        SHD_SRC_TC(64)
        default: return cudaErrorInvalidConfiguration;
    }
#undef SHD_SRC_TC
    note_launch();
    return cudaGetLastError();
}

}  // namespace shd
