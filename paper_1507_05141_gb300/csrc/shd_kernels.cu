// Kernels of one source iteration (stages a1..a5) for FP64 and FP32.
//
//   k_source    a2  comoving SH source with the group-to-group kernel
//   k_sweep     a4  short-characteristic transfer, plane by plane
// (a1 project and a3 sh2lab are in shd_transforms.cu)
//   k_sums_*    a5  FP64 diagnostics (deterministic two-pass reductions)
//
// Paper passages: Sec. 2 (eq:shdom, Lambda iteration, SH <-> DO transforms),
// Sec. 2.1 (eq:time), Sec. 2.2 (eq:lorentzfreq, eq:lorentzray, invariants,
// remap between frame meshes), Sec. 2.3 (SH source, Thomson, eq:comptoncross).
#include <cooperative_groups.h>
#include <cuda_runtime.h>

#include <cmath>
#include <vector>

#include "shd_internal.cuh"

namespace cg = cooperative_groups;

namespace shd {

template <class T>
Prob<T> make_prob(const shd_ctx *c)
{
    Prob<T> p;
    p.nx = c->nx; p.ny = c->ny; p.nz = c->nz; p.Nc = c->Nc;
    p.N = c->N; p.nmu = c->nmu; p.nphi = c->nphi; p.NLM = c->NLM; p.L = c->L; p.G = c->G;
    p.kappa = (T)c->kappa;
    p.ord = (const Ordinate *)c->d_ord;
    p.W = (const T *)c->d_W; p.dirs = (const T *)c->d_dirs; p.Y = (const T *)c->d_Y; p.mu = (const T *)c->d_mu;
    p.edges = c->d_edges; p.centre = c->d_centre;
    p.alpha0 = (const T *)c->d_alpha0; p.ne = (const T *)c->d_ne; p.u = (const T *)c->d_u;
    p.emis0 = (const T *)c->d_emis0; p.chi0 = (const T *)c->d_chi0;
    p.K = (const T *)c->d_K; p.sigma_out = (const T *)c->d_sigma_out;
    p.bc_mode = c->bc_mode; p.bc = (const T *)c->d_bc;
    p.tiles = (const TileInfo *)c->d_tiles; p.ntiles = c->ntiles;
    p.moving = c->d_moving; p.nmoving = c->nmoving; p.mflag = c->d_mflag;
    p.midx = c->d_midx; p.mtiles = c->d_mtiles; p.nmtiles = c->nmtiles;
    p.Bproj = (const T *)c->d_Bproj; p.NB = c->NB;
    p.fp64_boost = c->precision == SHD_MIXED ? 1 : 0;
    p.int2mesh = c->d_int2mesh; p.mesh2int = c->d_mesh2int; p.nA = c->nA;
    p.lc = (const T *)c->d_lc; p.linv = (const T *)c->d_linv;
    p.le0 = c->G ? (T)std::log(c->h_edges[0]) : T(0);
    p.leG = c->G ? (T)std::log(c->h_edges[c->G]) : T(0);
    p.lgu = c->lg_uniform ? 1 : 0;
    p.lgidl = (T)(1.0 / c->lg_dl);
    p.lgx0 = c->G ? (T)((std::log(c->h_edges[0]) - c->lg_c0) / c->lg_dl) : T(0);
    p.lgx1 = c->G ? (T)((std::log(c->h_edges[c->G]) - c->lg_c0) / c->lg_dl) : T(0);
    p.thermal = (c->scat_kind == SHD_SCAT_KN_THERMAL && c->have_theta && c->d_thK) ? 1 : 0;
    p.thb = c->d_thb;
    p.thw = (const T *)c->d_thw;
    p.thK = (const T *)c->d_thK;
    p.thso = (const T *)c->d_thso;
    p.thperm = c->d_thperm;
    p.thchunk = c->d_thchunk;
    p.nthchunk = c->nthchunk;
    return p;
}

__device__ inline void node_xyz(long long c, int nx, int ny, int &ix, int &iy, int &iz)
{
    ix = (int)(c % nx);
    long long r = c / nx;
    iy = (int)(r % ny);
    iz = (int)(r / ny);
}

// -------------------------------------------------------------------------
// chi0(c,g) = alpha0 + n_e sigma_out(g)  (Sec. 2: chi = alpha + sigma)
// -------------------------------------------------------------------------
template <class T>
__global__ void k_chi0(Prob<T> P, T *chi0)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    long long n = P.Nc * P.G;
    if (i >= n) return;
    long long c = i / P.G;
    int g = (int)(i % P.G);
    T so = P.sigma_out[g];
    if (P.thermal) {
        // the node's blend of its two bracketing temperature tables
        const int b = P.thb[c];
        const T w = P.thw[c];
        so = (T(1) - w) * P.thso[(size_t)b * P.G + g] + w * P.thso[(size_t)(b + 1) * P.G + g];
    }
    chi0[i] = P.alpha0[i] + P.ne[c] * so;
}

// chi0 in the three sweep layouts, chi0L[d][g][o] = chi0[c(o, d)][g]: at a
// node at rest the laboratory opacity of every ordinate is chi0 (Sec. 2.2
// with u = 0), so the sweep reads it from this small table instead of the
// per-ordinate chi_lab.
template <class T>
__global__ void k_chi0_layout(Prob<T> P, const T *__restrict__ chi0, T *__restrict__ chi0L, int *__restrict__ dirty)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const long long per = (long long)P.G * P.Nc;
    if (i >= 3 * per) return;
    const int d = (int)(i / per);
    const long long r = i - d * per;
    const int g = (int)(r / P.Nc);
    const long long o = r - (long long)g * P.Nc;
    int ix, iy, iz;
    if (d == 2) {  // (z, y, x)
        ix = (int)(o % P.nx); iy = (int)((o / P.nx) % P.ny); iz = (int)(o / ((long long)P.nx * P.ny));
    } else if (d == 1) {  // (y, z, x)
        ix = (int)(o % P.nx); iz = (int)((o / P.nx) % P.nz); iy = (int)(o / ((long long)P.nx * P.nz));
    } else {  // (x, z, y)
        iy = (int)(o % P.ny); iz = (int)((o / P.ny) % P.nz); ix = (int)(o / ((long long)P.ny * P.nz));
    }
    const long long c = ((long long)iz * P.ny + iy) * P.nx + ix;
    const T v = chi0[c * P.G + g];
    if (dirty && chi0L[i] != v) *dirty = 1;  // chi_lab at rest no longer holds chi0
    chi0L[i] = v;
}

// -------------------------------------------------------------------------
// a2: S_p(c,g) = n_e/chi0 sum_g' K_l[g][g'] I_p(c,g') + delta_p0 sqrt(4pi) eta0/chi0
// One CTA per node: the node's I_lm [G][NLM] is staged in shared memory
// (coalesced), every thread forms outputs of all groups from it.
// -------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_source(Prob<T> P, const T *__restrict__ Ip, T *__restrict__ Sp)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    T *sI = reinterpret_cast<T *>(smem_raw);  // [G][NLM]
    const int G = P.G, NLM = P.NLM;
    const long long c = blockIdx.x;
    const long long base = c * G * NLM;
    for (int i = threadIdx.x; i < G * NLM; i += blockDim.x) sI[i] = Ip[base + i];
    __syncthreads();
    const T ne = P.ne[c];
    for (int i = threadIdx.x; i < G * NLM; i += blockDim.x) {
        int g = i / NLM, p = i - g * NLM;
        int l = 0;
        while ((l + 1) * (l + 1) <= p) ++l;
        T chi = P.chi0[c * G + g];
        T s = T(0);
        if (chi > T(0)) {
            const T *Kr = P.K + ((size_t)l * G + g) * G;
            T acc = T(0);
            for (int gp = 0; gp < G; ++gp) acc += Kr[gp] * sI[gp * NLM + p];
            s = ne / chi * acc;
            if (p == 0) s += T(3.5449077018110320546) * P.emis0[c * G + g] / chi;  // sqrt(4 pi)
        }
        Sp[base + i] = s;
    }
}

// a2 + a5 fused for the stepping path: one warp per node (persistent grid of
// n_partial CTAs x 8 warps), the node's I_lm staged in the warp's shared
// tile, K_l in shared memory with rows padded against bank conflicts.  S_p
// is formed exactly as k_source forms it; while it is written, every thread
// accumulates in FP64 the residual |S - S_prev|^2, |S|^2 and, from J of the
// moments, the energy and photon sums; the CTA's partials go to partial[b][4]
// for k_sums_final.  DIAG: every K_l is diagonal (Thomson, isotropic), so an
// output takes one product and the node's I_lm streams straight through
// (the full sum's other terms are exact zeros: the same S_p).
template <class T, bool DIAG>
__global__ void __launch_bounds__(256, 3) k_source_sums(Prob<T> P, const T *__restrict__ Ip, T *__restrict__ Sp,
                                                     const T *__restrict__ mom, const T *__restrict__ Sprev,
                                                     int have_prev, double *partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][8];
    const int G = P.G, NLM = P.NLM, L = P.L;
    const int KS = G * G + 1;
    T *sK = reinterpret_cast<T *>(smem_raw);  // [L+1][KS]
    T *sI = sK + (((size_t)(L + 1) * KS + 1) & ~(size_t)1);  // [8][G][NLM]
    for (int i = threadIdx.x; i < (L + 1) * G * G; i += blockDim.x) {
        const int l = i / (G * G);
        sK[(size_t)l * KS + (i - l * G * G)] = P.K[i];
    }
    __syncthreads();
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *wI = sI + (size_t)warp * G * NLM;
    double e = 0, ph = 0, num = 0, den = 0;
    for (long long c = (long long)blockIdx.x * 8 + warp; c < P.Nc; c += (long long)gridDim.x * 8) {
        const long long base = c * G * NLM;
        const T ne = P.ne[c];
        if constexpr (DIAG) {
            // lane g < G holds group g's chi0, n_e/chi0 and emission term
            // (G <= 32 on this path), shared with the warp by shuffles
            const T chi_l = lane < G ? P.chi0[c * G + lane] : T(0);
            const T r_l = chi_l > T(0) ? ne / chi_l : T(0);
            const T em_l = chi_l > T(0) ? T(3.5449077018110320546) * P.emis0[c * G + lane] / chi_l : T(0);  // sqrt(4 pi)
            // the node's part of |S|^2 and |S - S_prev|^2 in working precision
            // (a lane's at most G ceil(NLM/32) squares), added to the FP64
            // totals once per node
            T dn = T(0), nm = T(0);
            // warp-uniform trip count: every lane takes part in the shuffles
            for (int p0 = 0; p0 < NLM; p0 += 32) {
                const int p = p0 + lane;
                const bool act = p < NLM;
                int l = 0;
                while ((l + 1) * (l + 1) <= p) ++l;
                // groups in rounds of 16: the round's loads are in flight together
                for (int g0 = 0; g0 < G; g0 += 16) {
                    T iv[16], pv[16];
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const long long i = base + (long long)(g0 + q) * NLM + p;
                        const bool ok = act && g0 + q < G;
                        iv[q] = ok ? Ip[i] : T(0);
                        pv[q] = ok && have_prev ? Sprev[i] : T(0);
                    }
#pragma unroll
                    for (int q = 0; q < 16; ++q) {
                        const int g = g0 + q;
                        if (g >= G) break;
                        const T chi = __shfl_sync(0xffffffffu, chi_l, g);
                        const T r = __shfl_sync(0xffffffffu, r_l, g);
                        const T em = __shfl_sync(0xffffffffu, em_l, g);
                        if (!act) continue;
                        T s = T(0);
                        if (chi > T(0)) {
                            T acc = T(0);
                            acc += sK[(size_t)l * KS + g * G + g] * iv[q];
                            s = r * acc;
                            if (p == 0) s += em;
                        }
                        Sp[base + (long long)g * NLM + p] = s;
                        dn += s * s;
                        if (have_prev) {
                            const T d = s - pv[q];
                            nm += d * d;
                        }
                    }
                }
            }
            den += (double)dn;
            num += (double)nm;
        } else {
        for (int i = lane; i < G * NLM; i += 32) wI[i] = Ip[base + i];
        __syncwarp();
        // the node's part of |S|^2 and |S - S_prev|^2 in working precision,
        // added to the FP64 totals once per node (an FP64 operation per
        // output would occupy the narrow FP64 pipe longer than the source)
        T dn = T(0), nm = T(0);
        for (int p = lane; p < NLM; p += 32) {
            int l = 0;
            while ((l + 1) * (l + 1) <= p) ++l;
            for (int g = 0; g < G; ++g) {
                const T chi = P.chi0[c * G + g];
                T s = T(0);
                if (chi > T(0)) {
                    const T *Kr = sK + (size_t)l * KS + g * G;
                    T acc = T(0);
                    for (int gp = 0; gp < G; ++gp) acc += Kr[gp] * wI[gp * NLM + p];
                    s = ne / chi * acc;
                    if (p == 0) s += T(3.5449077018110320546) * P.emis0[c * G + g] / chi;  // sqrt(4 pi)
                }
                const long long i = base + (long long)g * NLM + p;
                Sp[i] = s;
                dn += s * s;
                if (have_prev) {
                    const T d = s - Sprev[i];
                    nm += d * d;
                }
            }
        }
        den += (double)dn;
        num += (double)nm;
        }
        for (int g = lane; g < G; g += 32) {
            const double J = (double)mom[(c * G + g) * 10];
            const double de = P.edges[g + 1] - P.edges[g];
            e += 4.0 * kPi * J * de;
            ph += 4.0 * kPi * J * de / P.centre[g];
        }
        __syncwarp();
    }
    // fixed-order reduction: lanes by shuffle, then the 8 warps
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, o);
        ph += __shfl_down_sync(0xffffffffu, ph, o);
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if (lane == 0) {
        red[0][warp] = e;
        red[1][warp] = ph;
        red[2][warp] = num;
        red[3][warp] = den;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double acc = 0;
        for (int w = 0; w < 8; ++w) acc += red[threadIdx.x][w];
        partial[blockIdx.x * 4 + threadIdx.x] = acc;
    }
}

// asynchronous copy of BYTES (4, 8 or 16) from global to shared memory
template <int BYTES>
__device__ inline void cp_async_n(void *smem, const void *gmem)
{
    unsigned sa = (unsigned)__cvta_generic_to_shared(smem);
    if constexpr (BYTES == 16)
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(sa), "l"(gmem));
    else
        asm volatile("cp.async.ca.shared.global [%0], [%1], %2;\n" ::"r"(sa), "l"(gmem), "n"(BYTES));
}

// -------------------------------------------------------------------------
// a2 + a5 for kernels that mix groups (Klein-Nishina, any non-diagonal
// table), FP32: per l the dense contraction S_l[g][(c, m)] = n_e/chi0 sum_g'
// K_l[g][g'] I_l[g'][(c, m)] (Sec. 2.3, eq:source) on the CUDA cores,
// register-blocked.  A unit is (l, group block of 4, m); a thread holds its
// unit's 4 groups x TN nodes of one harmonic p and, per g', takes the four
// K_l[g][g'] in one 16-byte load (K stored [l][g'][g]) and the TN values
// I[c][g'][p] as broadcasts: 32 FMAs a 9 loads at TN = 8.  Units run
// l-major, m fastest, so the lanes of a warp share a K row.  Tiles of TN
// consecutive nodes (one contiguous [TN][G][NLM] block of I_lm, and the
// same block of S_prev for the residual) stream through a two-stage
// cp.async ring; the CTA is persistent over tiles.  The
// residual parts |S|^2, |S - S_prev|^2 accumulate per unit in FP32 and join
// the FP64 totals once per unit; the energy and photon sums stay FP64.
// -------------------------------------------------------------------------
template <int TN, bool PS>
__global__ void __launch_bounds__(512, 1) k_source_kn(Prob<float> P, const float *__restrict__ Ip,
                                                      float *__restrict__ Sp, const float *__restrict__ mom,
                                                      const float *__restrict__ Sprev, int have_prev,
                                                      double *partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][16];
    const int G = P.G, NLM = P.NLM, L = P.L;
    const int Gb = (G + 3) / 4, G4 = 4 * Gb;
    const int tile_f = TN * G * NLM;  // floats of one tile of I_lm
    float *sK = reinterpret_cast<float *>(smem_raw);  // [L+1][G][G4]: K_l[g][g'] at [l][g'][g]
    float *sI = sK + (size_t)(L + 1) * G * G4;        // [2][TN][G][NLM]
    float *sP = sI + (size_t)2 * tile_f;              // PS: [2][TN][G][NLM] S_prev of the tile
    float *sR = sP + (PS ? (size_t)2 * tile_f : 0);   // [TN][G4] n_e/chi0 (0 where chi0 <= 0)
    float *sE = sR + TN * G4;                         // [TN][G4] sqrt(4 pi) eta0/chi0
    const int tid = threadIdx.x, nt = blockDim.x;
    for (int i = tid; i < (L + 1) * G * G4; i += nt) {
        const int l = i / (G * G4), rem = i - l * G * G4, gp = rem / G4, g = rem - gp * G4;
        sK[i] = g < G ? P.K[((size_t)l * G + g) * G + gp] : 0.f;
    }
    const long long ntile = (P.Nc + TN - 1) / TN;
    auto load = [&](long long t, int buf) {
        if (t < ntile) {
            const long long c0 = t * TN;
            const int nn = (int)(P.Nc - c0 < TN ? P.Nc - c0 : TN);
            const int nv = nn * G * NLM / 4;  // 16-byte pieces (G NLM is a multiple of 4)
            const float *src = Ip + c0 * G * NLM;
            float *dst = sI + (size_t)buf * tile_f;
            for (int q = tid; q < nv; q += nt) cp_async_n<16>(dst + 4 * q, src + 4 * q);
            if (PS && have_prev) {  // the tile's S_prev, read by the epilogue
                const float *sp = Sprev + c0 * G * NLM;
                float *dp = sP + (size_t)buf * tile_f;
                for (int q = tid; q < nv; q += nt) cp_async_n<16>(dp + 4 * q, sp + 4 * q);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };
    double e = 0, ph = 0, num = 0, den = 0;
    const int nunit = Gb * NLM;
    load(blockIdx.x, 0);
    int it = 0;
    for (long long t = blockIdx.x; t < ntile; t += gridDim.x, ++it) {
        const int buf = it & 1;
        const long long c0 = t * TN;
        const int nn = (int)(P.Nc - c0 < TN ? P.Nc - c0 : TN);
        asm volatile("cp.async.wait_group 0;\n" ::);
        __syncthreads();  // this tile's I_lm landed; the previous tile's reads of sR, sE and its buffer are done
        load(t + gridDim.x, buf ^ 1);
        for (int i = tid; i < TN * G4; i += nt) {
            const int n = i / G4, g = i - n * G4;
            float r = 0.f, em = 0.f;
            if (n < nn && g < G) {
                const long long c = c0 + n;
                const float chi = P.chi0[c * G + g];
                if (chi > 0.f) {
                    r = P.ne[c] / chi;
                    em = 3.5449077018110320546f * P.emis0[c * G + g] / chi;  // sqrt(4 pi)
                }
            }
            sR[i] = r;
            sE[i] = em;
        }
        for (int i = tid; i < nn * G; i += nt) {
            const int g = i % G;
            const double J = (double)mom[(c0 * G + i) * 10];
            const double de = P.edges[g + 1] - P.edges[g];
            e += 4.0 * kPi * J * de;
            ph += 4.0 * kPi * J * de / P.centre[g];
        }
        __syncthreads();
        const float *tI = sI + (size_t)buf * tile_f;
        const float *tP = sP + (size_t)buf * tile_f;
        for (int u = tid; u < nunit; u += nt) {
            // unit u: band l holds the Gb (2l + 1) units from Gb l^2 on
            int l = (int)sqrtf((float)(u / Gb));
            while (Gb * (l + 1) * (l + 1) <= u) ++l;
            while (Gb * l * l > u) --l;
            const int r = u - Gb * l * l, gb = r / (2 * l + 1), p = l * l + (r - gb * (2 * l + 1));
            float acc[4][TN];
#pragma unroll
            for (int j = 0; j < 4; ++j)
#pragma unroll
                for (int n = 0; n < TN; ++n) acc[j][n] = 0.f;
            const float4 *kr = reinterpret_cast<const float4 *>(sK + (size_t)l * G * G4) + gb;
            const float *ir = tI + p;
#pragma unroll 4
            for (int gp = 0; gp < G; ++gp) {
                const float4 k4 = kr[(size_t)gp * Gb];
                float iv[TN];
#pragma unroll
                for (int n = 0; n < TN; ++n) iv[n] = ir[((size_t)n * G + gp) * NLM];
#pragma unroll
                for (int n = 0; n < TN; ++n) {
                    acc[0][n] += k4.x * iv[n];
                    acc[1][n] += k4.y * iv[n];
                    acc[2][n] += k4.z * iv[n];
                    acc[3][n] += k4.w * iv[n];
                }
            }
            // per group of the unit: its TN outputs and S_prev (PS: the
            // tile's, in shared memory; else TN predicated loads in flight
            // together), then the stores and the residual parts
            float dn = 0.f, nmr = 0.f;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int g = 4 * gb + j;
                const bool gv = g < G;
                const long long ob = ((c0 * G + g) * NLM + p);  // node n adds n G NLM
                float sv[TN], pv[TN];
#pragma unroll
                for (int n = 0; n < TN; ++n) {
                    sv[n] = sR[n * G4 + g] * acc[j][n];
                    if (p == 0) sv[n] += sE[n * G4 + g];
                    pv[n] = 0.f;
                }
                if (have_prev) {
#pragma unroll
                    for (int n = 0; n < TN; ++n)
                        if (gv && n < nn)
                            pv[n] = PS ? tP[((size_t)n * G + g) * NLM + p] : Sprev[ob + (long long)n * G * NLM];
                }
#pragma unroll
                for (int n = 0; n < TN; ++n) {
                    if (gv && n < nn) {
                        Sp[ob + (long long)n * G * NLM] = sv[n];
                        dn += sv[n] * sv[n];
                        const float d = sv[n] - pv[n];
                        if (have_prev) nmr += d * d;
                    }
                }
            }
            den += (double)dn;
            num += (double)nmr;
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    // fixed-order reduction: lanes by shuffle, then the warps
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, o);
        ph += __shfl_down_sync(0xffffffffu, ph, o);
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if (lane == 0) {
        red[0][warp] = e;
        red[1][warp] = ph;
        red[2][warp] = num;
        red[3][warp] = den;
    }
    __syncthreads();
    if (tid < 4) {
        double a = 0;
        for (int w = 0; w < nw; ++w) a += red[tid][w];
        partial[blockIdx.x * 4 + tid] = a;
    }
}

// -------------------------------------------------------------------------
// a4: one CTA per (ordinate, group).  Planes normal to the dominant axis are
// contiguous in the sweep layout and depend only on the previous plane, so
// the CTA walks them in upwind order holding the previous plane's I^{n+1},
// S~ and chi~ in shared memory; each thread keeps its own nodes' values in
// registers between the two barriers of a plane.
// -------------------------------------------------------------------------
template <class T, int NPT>
__global__ void __launch_bounds__(1024) k_sweep(Prob<T> P, T *__restrict__ I, const T *__restrict__ eta,
                                                const T *__restrict__ chi)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int k = blockIdx.x / P.G;
    const int g = blockIdx.x - k * P.G;
    const Ordinate o = P.ord[k];
    const int dims[3] = {P.nx, P.ny, P.nz};
    const int nd = dims[o.d], n1 = dims[o.e1], n2 = dims[o.e2];
    const int plane = n1 * n2;
    T *pI = reinterpret_cast<T *>(smem_raw);
    T *pS = pI + plane;
    T *pC = pS + plane;
    const long long base = ((long long)k * P.G + g) * P.Nc;
    const T fr1 = (T)o.fr1, fr2 = (T)o.fr2, s = (T)o.s, kap = P.kappa;
    const int first1 = o.s1 > 0 ? 0 : n1 - 1, first2 = o.s2 > 0 ? 0 : n2 - 1;
    const T w00 = (T(1) - fr1) * (T(1) - fr2), w10 = fr1 * (T(1) - fr2), w01 = (T(1) - fr1) * fr2, w11 = fr1 * fr2;
    T bc_iso = P.bc_mode == SHD_BC_ISO ? P.bc[g] : T(0);

    T rI[NPT], rS[NPT], rC[NPT];
    for (int step = 0; step < nd; ++step) {
        const int id = o.sd > 0 ? step : nd - 1 - step;
        const long long pbase = base + (long long)id * plane;
#pragma unroll
        for (int t = 0; t < NPT; ++t) {
            int j = threadIdx.x + t * blockDim.x;
            if (j >= plane) break;
            int i1 = j / n2, i2 = j - i1 * n2;
            long long oo = pbase + j;
            T In = I[oo];
            T ct = chi[oo] + kap;
            T st = ct > T(0) ? (eta[oo] + kap * In) / ct : T(0);
            bool inflow = step == 0 || (o.s1 != 0 && i1 == first1) || (o.s2 != 0 && i2 == first2);
            T inew;
            if (inflow) {
                inew = P.bc_mode == SHD_BC_FULL ? P.bc[oo] : bc_iso;
            } else {
                int j1 = i1 - o.s1, j2 = i2 - o.s2;  // upwind neighbours on the previous plane
                int a00 = i1 * n2 + i2, a10 = j1 * n2 + i2, a01 = i1 * n2 + j2, a11 = j1 * n2 + j2;
                // a zero weight may pair with an index outside the plane when the
                // component is zero; clamp it to a valid slot (its weight is 0)
                if (o.s1 == 0) { a10 = a00; a11 = a01; }
                if (o.s2 == 0) { a01 = a00; a11 = a10; }
                T iu = w00 * pI[a00] + w10 * pI[a10] + w01 * pI[a01] + w11 * pI[a11];
                T su = w00 * pS[a00] + w10 * pS[a10] + w01 * pS[a01] + w11 * pS[a11];
                T cu = w00 * pC[a00] + w10 * pC[a10] + w01 * pC[a01] + w11 * pC[a11];
                T dtau = s * T(0.5) * (cu + ct);
                T e, wp, wu;
                sc_weights<T>(dtau, e, wp, wu);
                inew = iu * e + st * wp + su * wu;
            }
            rI[t] = inew;
            rS[t] = st;
            rC[t] = ct;
        }
        __syncthreads();
#pragma unroll
        for (int t = 0; t < NPT; ++t) {
            int j = threadIdx.x + t * blockDim.x;
            if (j >= plane) break;
            pI[j] = rI[t];
            pS[j] = rS[t];
            pC[j] = rC[t];
            I[pbase + j] = rI[t];
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------------
// a4, pipelined: the same plane walk with the inputs of the next plane
// (I^n, eta_lab, chi_lab) already streaming into a two-stage shared-memory
// ring by cp.async (16-byte pieces when aligned) while the current plane is
// computed.  Lane i of a warp owns node j = tid + 1024 u of every plane, so
// every shared-memory access of a warp is to consecutive words (no bank
// conflicts) and every global access is coalesced; the node's in-plane
// upwind neighbours and inflow flags are computed once.  Two barriers per
// plane: after the copies land (they and the previous plane's state become
// visible) and after the reads of the previous plane.
// -------------------------------------------------------------------------
template <class T>
__device__ inline T fast_recip(T x);
template <>
__device__ inline double fast_recip<double>(double x) { return 1.0 / x; }
template <>
__device__ inline float fast_recip<float>(float x) { return hw_rcp(x); }


// With `mbits` (16-byte copies only), chi comes from the per-ordinate chi_lab
// only for the 4-node pieces of a plane that hold a moving node (bit id % 64
// of mbits[d][id / 64][piece]) and from chi0L elsewhere; the CTA keeps the
// current 64-plane window of its layout's bits in shared memory.
// WIDE: the transfer weights switch to FP64 above optical depth kFp64Tau
// (launched unless the host bound excludes such steps).
template <class T, int U, bool VEC, bool CB, bool WIDE>
__global__ void __launch_bounds__(1024, 1) k_sweep_pipe(Prob<T> P, T *__restrict__ I, const T *__restrict__ eta,
                                                        const T *__restrict__ chi, const T *__restrict__ chi0L,
                                                        const unsigned long long *__restrict__ mbits, int npc,
                                                        int nwin)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NT = 1024;
    constexpr int V = 16 / sizeof(T);  // reals per 16-byte copy
    const int k = blockIdx.x / P.G;
    const int g = blockIdx.x - k * P.G;
    const Ordinate o = P.ord[k];
    const int dims[3] = {P.nx, P.ny, P.nz};
    const int nd = dims[o.d], n1 = dims[o.e1], n2 = dims[o.e2];
    const int plane = n1 * n2;
    const int pstride = (int)(((size_t)plane + 3) & ~(size_t)3);  // keep every array 16-byte aligned
    // previous plane: FP32 keeps (I, S, chi) of a node in one float4, FP64
    // keeps I apart from the (S, chi) pairs
    constexpr bool PK = sizeof(T) == 4;
    using T2 = typename std::conditional<sizeof(T) == 4, float2, double2>::type;
    float4 *pQ = reinterpret_cast<float4 *>(smem_raw);
    T *pI = reinterpret_cast<T *>(smem_raw);
    T2 *pSC = reinterpret_cast<T2 *>(pI + pstride);
    T *ring = pI + (PK ? 4 : 3) * pstride;  // [2][3][pstride]
    unsigned long long *sbits = reinterpret_cast<unsigned long long *>(ring + 6 * pstride);  // [npc]
    const long long base = ((long long)k * P.G + g) * P.Nc;
    constexpr bool cbits = VEC && CB;
    const T *c0base = cbits ? chi0L + ((long long)o.d * P.G + g) * P.Nc : nullptr;
    const T fr1 = (T)o.fr1, fr2 = (T)o.fr2, s = (T)o.s, kap = P.kappa;
    const T w00 = (T(1) - fr1) * (T(1) - fr2), w10 = fr1 * (T(1) - fr2), w01 = (T(1) - fr1) * fr2, w11 = fr1 * fr2;
    const T bc_iso = P.bc_mode == SHD_BC_ISO ? P.bc[g] : T(0);
    const bool bc_full = P.bc_mode == SHD_BC_FULL;
    const int tid = threadIdx.x;

    // node j = tid + NT*u of every plane; bit u of `face` marks an inflow
    // face of one of the two in-plane axes; the upwind neighbours on the
    // previous plane are j - d1, j - d2, j - d1 - d2
    unsigned face = 0;
    {
        const int first1 = o.s1 > 0 ? 0 : n1 - 1, first2 = o.s2 > 0 ? 0 : n2 - 1;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int j = tid + NT * u;
            int i1 = j / n2, i2 = j - i1 * n2;
            if ((o.s1 != 0 && i1 == first1) || (o.s2 != 0 && i2 == first2)) face |= 1u << u;
        }
    }
    const int d1 = o.s1 * n2, d2 = o.s2;

    auto issue = [&](int step) {
        if (step < nd) {
            const int id = o.sd > 0 ? step : nd - 1 - step;
            const long long pb = base + (long long)id * plane;
            T *r = ring + (size_t)(step & 1) * 3 * pstride;
            if constexpr (VEC) {
                const int nv = plane / V;  // 16-byte pieces per array
                for (int q = tid; q < nv; q += NT) cp_async_n<16>(&r[q * V], &I[pb + q * V]);
                for (int q = tid; q < nv; q += NT) cp_async_n<16>(&r[pstride + q * V], &eta[pb + q * V]);
                for (int q = tid; q < nv; q += NT) {
                    const int off = q * V;
                    const T *src = chi + pb + off;
                    if (cbits && !((sbits[off >> 2] >> (id & 63)) & 1ull)) src = c0base + (long long)id * plane + off;
                    cp_async_n<16>(&r[2 * pstride + off], src);
                }
            } else {
#pragma unroll
                for (int u = 0; u < U; ++u) {
                    const int j = tid + NT * u;
                    if (j >= plane) break;
                    cp_async_n<sizeof(T)>(&r[j], &I[pb + j]);
                    cp_async_n<sizeof(T)>(&r[pstride + j], &eta[pb + j]);
                    cp_async_n<sizeof(T)>(&r[2 * pstride + j], &chi[pb + j]);
                }
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };

    // the window of moving-piece bits that holds plane `step`
    int cur_w = -1;
    auto window = [&](int step) {
        if (!cbits || step >= nd) return;
        const int w = (o.sd > 0 ? step : nd - 1 - step) >> 6;
        if (w == cur_w) return;
        for (int i = tid; i < npc; i += NT) sbits[i] = mbits[((size_t)o.d * nwin + w) * npc + i];
        cur_w = w;
        __syncthreads();
    };

    window(0);
    issue(0);
    T rI[U], rS[U], rC[U];
    for (int step = 0; step < nd; ++step) {
        asm volatile("cp.async.wait_group 0;\n" ::);
        __syncthreads();  // every copy of this plane and the previous plane's state are visible
        window(step + 1);
        issue(step + 1);
        const T *r = ring + (size_t)(step & 1) * 3 * pstride;
        const bool first = step == 0;
        const int id = o.sd > 0 ? step : nd - 1 - step;
        const long long pb = base + (long long)id * plane;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = tid + NT * u;
            if (j >= plane) break;
            const T In = r[j];
            const T ct = r[2 * pstride + j] + kap;
            const T st = ct > T(0) ? (r[pstride + j] + kap * In) * fast_recip<T>(ct) : T(0);
            T inew;
            if (first || ((face >> u) & 1u)) {
                inew = bc_full ? P.bc[pb + j] : bc_iso;
            } else {
                const int b00 = j, b10 = j - d1, b01 = j - d2, b11 = j - d1 - d2;
                T iu, su, cu;
                if constexpr (PK) {
                    const float4 q00 = pQ[b00], q10 = pQ[b10], q01 = pQ[b01], q11 = pQ[b11];
                    iu = w00 * q00.x + w10 * q10.x + w01 * q01.x + w11 * q11.x;
                    su = w00 * q00.y + w10 * q10.y + w01 * q01.y + w11 * q11.y;
                    cu = w00 * q00.z + w10 * q10.z + w01 * q01.z + w11 * q11.z;
                } else {
                    iu = w00 * pI[b00] + w10 * pI[b10] + w01 * pI[b01] + w11 * pI[b11];
                    const T2 q00 = pSC[b00], q10 = pSC[b10], q01 = pSC[b01], q11 = pSC[b11];
                    su = w00 * q00.x + w10 * q10.x + w01 * q01.x + w11 * q11.x;
                    cu = w00 * q00.y + w10 * q10.y + w01 * q01.y + w11 * q11.y;
                }
                const T dtau = s * T(0.5) * (cu + ct);
                T ew, wp, wu;
                if constexpr (WIDE) sc_weights<T>(dtau, ew, wp, wu);
                else sc_weights_narrow<T>(dtau, ew, wp, wu);
                inew = iu * ew + st * wp + su * wu;
            }
            rI[u] = inew;
            rS[u] = st;
            rC[u] = ct;
        }
        __syncthreads();  // all reads of the previous plane are done
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = tid + NT * u;
            if (j >= plane) break;
            if constexpr (PK) {
                pQ[j] = make_float4(rI[u], rS[u], rC[u], 0.f);
            } else {
                pI[j] = rI[u];
                T2 q;
                q.x = rS[u];
                q.y = rC[u];
                pSC[j] = q;
            }
            I[pb + j] = rI[u];
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}

// -------------------------------------------------------------------------
// a4, FP32 with two previous-plane buffers: plane s reads the state of plane
// s-1 from one float4 buffer (I, S, chi of a node) and writes its own into
// the other, so one barrier per plane suffices: it makes plane s-1's state
// and the copies of plane s visible, and every read of the buffer plane s
// overwrites (plane s-2's) is done by then.  The inputs of plane s+1 stream
// into a two-stage ring as in k_sweep_pipe (16-byte copies; a plane that
// does not start on a 16-byte boundary is copied as its aligned cover and
// read from its offset in the slot, so grids of any size keep the 16-byte
// copies); with CB (aligned planes only) the moving-piece bits are read
// from global memory when a plane's copies are issued.
// -------------------------------------------------------------------------
// One (ordinate, group) pair of the plane sweep by the CTA (tune_stride > 0,
// schedule timing only: into column blockIdx.x of a scratch intensity).
// reals by which p lies past the 16-byte boundary below it (p 4-byte aligned)
__device__ __forceinline__ int shift16(const float *p)
{
    return (int)((reinterpret_cast<unsigned long long>(p) >> 2) & 3ull);
}

template <int U, bool CB, bool WIDE, int NT = 1024>
__device__ __forceinline__ void sweep_pair_pp(const Prob<float> &P, float *__restrict__ I,
                                              const float *__restrict__ eta, const float *__restrict__ chi,
                                              const float *__restrict__ chi0L,
                                              const unsigned long long *__restrict__ mbits, int npc, int nwin,
                                              int pair, int tune_stride, unsigned char *smem_raw)
{
    const int k = pair / P.G;
    const int g = pair - k * P.G;
    const Ordinate o = P.ord[k];
    const int dims[3] = {P.nx, P.ny, P.nz};
    const int nd = dims[o.d], n1 = dims[o.e1], n2 = dims[o.e2];
    const int plane = n1 * n2;
    // planes whose start is not 16-byte aligned (grids with a plane or Nc
    // not a multiple of 4) are copied as their aligned cover, up to 3 reals
    // on either side: 4 reals of room past the rounded plane
    const int pstride = ((plane + 3) & ~3) + 4;
    float4 *Q = reinterpret_cast<float4 *>(smem_raw);              // [2][pstride]
    float *ring = reinterpret_cast<float *>(Q + 2 * (size_t)pstride);  // [2][3][pstride]
    const long long base = ((long long)k * P.G + g) * P.Nc;
    if (tune_stride > 0) I += (long long)blockIdx.x * P.Nc - base;
    const float *c0base = CB ? chi0L + ((long long)o.d * P.G + g) * P.Nc : nullptr;
    const unsigned long long *mb = CB ? mbits + (size_t)o.d * nwin * npc : nullptr;
    const float fr1 = (float)o.fr1, fr2 = (float)o.fr2, s = (float)o.s, kap = P.kappa;
    const float w00 = (1.f - fr1) * (1.f - fr2), w10 = fr1 * (1.f - fr2), w01 = (1.f - fr1) * fr2, w11 = fr1 * fr2;
    const float bc_iso = P.bc_mode == SHD_BC_ISO ? P.bc[g] : 0.f;
    const bool bc_full = P.bc_mode == SHD_BC_FULL;
    const int tid = threadIdx.x;

    unsigned face = 0;
    {
        const int first1 = o.s1 > 0 ? 0 : n1 - 1, first2 = o.s2 > 0 ? 0 : n2 - 1;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            int j = tid + NT * u;
            int i1 = j / n2, i2 = j - i1 * n2;
            if ((o.s1 != 0 && i1 == first1) || (o.s2 != 0 && i2 == first2)) face |= 1u << u;
        }
    }
    const int d1 = o.s1 * n2, d2 = o.s2;
    // the moving-node bits of this thread's chi pieces (plane <= U NT nodes,
    // 4 a piece: at most MP pieces a thread) for the current 64-plane
    // window, held in registers and reloaded when the window changes
    constexpr int MP = (U + 3) / 4;
    unsigned long long mw[MP];
    int mwin = -1;

    auto issue = [&](int step) {
        if (step < nd) {
            const int id = o.sd > 0 ? step : nd - 1 - step;
            const long long pb = base + (long long)id * plane;
            float *r = ring + (size_t)(step & 1) * 3 * pstride;
            if constexpr (!CB) {
                // the aligned cover of the plane in each array, shifted by
                // the start's offset a within its 16 bytes (reals [a, a+plane)
                // of the slot hold the plane)
                const int aI = shift16(I + pb), aE = shift16(eta + pb), aC = shift16(chi + pb);
                const float *gI = I + pb - aI, *gE = eta + pb - aE, *gC = chi + pb - aC;
                const int nI = (aI + plane + 3) >> 2, nE = (aE + plane + 3) >> 2, nC = (aC + plane + 3) >> 2;
                for (int q = tid; q < nI; q += NT) cp_async_n<16>(&r[q * 4], gI + q * 4);
                for (int q = tid; q < nE; q += NT) cp_async_n<16>(&r[pstride + q * 4], gE + q * 4);
                for (int q = tid; q < nC; q += NT) cp_async_n<16>(&r[2 * pstride + q * 4], gC + q * 4);
                asm volatile("cp.async.commit_group;\n" ::);
                return;
            }
            const int nv = plane / 4;  // 16-byte pieces per array (aligned planes)
            for (int q = tid; q < nv; q += NT) cp_async_n<16>(&r[q * 4], &I[pb + q * 4]);
            for (int q = tid; q < nv; q += NT) cp_async_n<16>(&r[pstride + q * 4], &eta[pb + q * 4]);
            if (CB && (id >> 6) != mwin) {
                mwin = id >> 6;
#pragma unroll
                for (int pi = 0; pi < MP; ++pi) {
                    const int q = tid + pi * NT;
                    mw[pi] = q < nv ? mb[(size_t)mwin * npc + q] : 0ull;
                }
            }
#pragma unroll
            for (int pi = 0; pi < MP; ++pi) {
                const int q = tid + pi * NT;
                if (q >= nv) break;
                const int off = q * 4;
                const float *src = chi + pb + off;
                if (CB && !((mw[pi] >> (id & 63)) & 1ull)) src = c0base + (long long)id * plane + off;
                cp_async_n<16>(&r[2 * pstride + off], src);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };

    issue(0);
    for (int step = 0; step < nd; ++step) {
        asm volatile("cp.async.wait_group 0;\n" ::);
        __syncthreads();  // this plane's copies and the previous plane's state are visible
        issue(step + 1);
        const bool first = step == 0;
        const int id = o.sd > 0 ? step : nd - 1 - step;
        const long long pb = base + (long long)id * plane;
        // per-plane bases of this thread's accesses: node u of the thread is
        // at a constant offset NT u from each (the upwind ones are formed for
        // every node but read only off the inflow faces)
        const float *rI = ring + (size_t)(step & 1) * 3 * pstride + tid;
        const float *rE = rI + pstride, *rC = rI + 2 * pstride;
        if constexpr (!CB) {
            rI += shift16(I + pb);
            rE += shift16(eta + pb);
            rC += shift16(chi + pb);
        }
        const float4 *qa = Q + (size_t)((step + 1) & 1) * pstride + tid;  // plane step - 1
        const float4 *qb = qa - d1, *qc = qa - d2, *qd = qa - d1 - d2;
        float4 *qn = Q + (size_t)(step & 1) * pstride + tid;               // plane step
        float *ig = I + pb + tid;
        const unsigned bnd = first ? ~0u : face;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            if (tid + NT * u >= plane) break;
            const float In = rI[NT * u];
            const float ct = rC[NT * u] + kap;
            const float st = ct > 0.f ? (rE[NT * u] + kap * In) * hw_rcp(ct) : 0.f;
            float inew;
            if ((bnd >> u) & 1u) {
                inew = bc_full ? P.bc[pb + tid + NT * u] : bc_iso;
            } else {
                const float4 q00 = qa[NT * u], q10 = qb[NT * u], q01 = qc[NT * u], q11 = qd[NT * u];
                const float iu = w00 * q00.x + w10 * q10.x + w01 * q01.x + w11 * q11.x;
                const float su = w00 * q00.y + w10 * q10.y + w01 * q01.y + w11 * q11.y;
                const float cu = w00 * q00.z + w10 * q10.z + w01 * q01.z + w11 * q11.z;
                const float dtau = s * 0.5f * (cu + ct);
                float ew, wp, wu;
                if constexpr (WIDE) sc_weights<float>(dtau, ew, wp, wu);
                else sc_weights_narrow_x2(dtau, ew, wp, wu);
                inew = iu * ew + st * wp + su * wu;
            }
            qn[NT * u] = make_float4(inew, st, ct, 0.f);
            ig[NT * u] = inew;
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
}

// NT threads a CTA (1024, or 512 / 256 for small planes, 1024 / NT CTAs
// an SM at the same 64 registers a thread)
template <int U, bool CB, bool WIDE, int NT>
__global__ void __launch_bounds__(NT, 1024 / NT) k_sweep_pp(Prob<float> P, float *__restrict__ I,
                                                      const float *__restrict__ eta, const float *__restrict__ chi,
                                                      const float *__restrict__ chi0L,
                                                      const unsigned long long *__restrict__ mbits, int npc, int nwin,
                                                      int tune_stride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    // tune_stride > 0 (schedule timing only): CTA b sweeps pair b * tune_stride
    // with its intensity in column b of a scratch array I [b][Nc]
    const int pair = tune_stride > 0 ? (int)blockIdx.x * tune_stride : (int)blockIdx.x;
    sweep_pair_pp<U, CB, WIDE, NT>(P, I, eta, chi, chi0L, mbits, npc, nwin, pair, tune_stride, smem_raw);
}

// The plane sweeps of a batch of problems in one persistent launch: CTAs
// walk the work list of every problem's (ordinate, group) pairs (problem p
// owns items [item0, item0 + N G)), each item as k_sweep_pp sweeps it, with
// the problem's own fields and arrays.  One launch per class of problems
// that share the kernel's variant (U, CB, WIDE).
template <int U, bool CB, bool WIDE>
__global__ void __launch_bounds__(1024, 1) k_sweep_batch(const SweepBatchProb *__restrict__ bp, int nprob,
                                                         long long nitems)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    for (long long it = blockIdx.x; it < nitems; it += gridDim.x) {
        int lo = 0, hi = nprob - 1;  // the last problem whose first item is <= it
        while (lo < hi) {
            const int mid = (lo + hi + 1) >> 1;
            if (bp[mid].item0 <= it) lo = mid;
            else hi = mid - 1;
        }
        const SweepBatchProb &b = bp[lo];
        __syncthreads();  // the previous item's reads of the shared buffers are done
        sweep_pair_pp<U, CB, WIDE>(b.P, b.I, b.eta, b.chi, b.chi0L, b.mbits, b.npc, b.nwin, (int)(it - b.item0), 0,
                                   smem_raw);
    }
}

// -------------------------------------------------------------------------
// a4, FP32, one plane split over a cluster of C CTAs: CTA r of the cluster
// owns rows [r R, r R + R) of the plane (R rows of the in-plane axis e1, a
// contiguous block of the sweep layout) and keeps the two previous-plane
// buffers of k_sweep_pp for them only.  Upwind neighbours one row back that
// belong to the neighbouring CTA (the first row of a CTA when n sweeps
// towards +e1, the last when towards -e1) are read from that CTA's buffer
// through distributed shared memory.  One cluster barrier per plane orders
// the buffers exactly as k_sweep_pp's block barrier does, now across the
// cluster.  Smaller CTAs let two or more clusters share an SM, so one
// cluster's barrier wait overlaps another's compute; planes larger than one
// CTA's shared memory fit across the cluster.  Every CTA runs every barrier
// (no early exit) and a final one keeps its buffers alive until the peers'
// last reads are done.  At 384 threads (three nodes a thread) the register
// cap is 56, so three CTAs share an SM: one more cluster's compute under
// each barrier wait.
// -------------------------------------------------------------------------
template <int U, bool CB, bool WIDE, int NT>
__global__ void __launch_bounds__(NT, NT == 384 ? 3 : 1024 / NT) k_sweep_cl(Prob<float> P, float *__restrict__ I, const float *__restrict__ eta,
                                                 const float *__restrict__ chi, const float *__restrict__ chi0L,
                                                 const unsigned long long *__restrict__ mbits, int npc, int nwin,
                                                 int pstride, int tune_stride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    cg::cluster_group cl = cg::this_cluster();
    const int C = (int)cl.num_blocks();
    const int r = (int)cl.block_rank();
    // tune_stride > 0 (schedule timing only): cluster b sweeps pair b *
    // tune_stride with its intensity in column b of a scratch array I [b][Nc]
    const int cidx = (int)blockIdx.x / C;
    const int pair = tune_stride > 0 ? cidx * tune_stride : cidx;
    const int k = pair / P.G;
    const int g = pair - k * P.G;
    const Ordinate o = P.ord[k];
    const int dims[3] = {P.nx, P.ny, P.nz};
    const int nd = dims[o.d], n1 = dims[o.e1], n2 = dims[o.e2];
    const int plane = n1 * n2;
    // rows per CTA: ceil(n1 / C), rounded up so every CTA's block of the
    // layout starts on a 16-byte boundary
    int R = (n1 + C - 1) / C;
    const int q4 = (n2 & 3) == 0 ? 1 : ((n2 & 1) == 0 ? 2 : 4);
    R = (R + q4 - 1) / q4 * q4;
    const int row0 = r * R;
    const int nrows = row0 >= n1 ? 0 : (n1 - row0 < R ? n1 - row0 : R);
    const int nloc = nrows * n2;
    const int j0 = row0 * n2;
    float4 *Q = reinterpret_cast<float4 *>(smem_raw);                  // [2][pstride]
    float *ring = reinterpret_cast<float *>(Q + 2 * (size_t)pstride);  // [2][3][pstride]
    const long long base = ((long long)k * P.G + g) * P.Nc;
    if (tune_stride > 0) I += (long long)cidx * P.Nc - base;
    const float *c0base = CB ? chi0L + ((long long)o.d * P.G + g) * P.Nc : nullptr;
    const unsigned long long *mb = CB ? mbits + (size_t)o.d * nwin * npc : nullptr;
    const float fr1 = (float)o.fr1, fr2 = (float)o.fr2, s = (float)o.s, kap = P.kappa;
    const float w00 = (1.f - fr1) * (1.f - fr2), w10 = fr1 * (1.f - fr2), w01 = (1.f - fr1) * fr2, w11 = fr1 * fr2;
    const float bc_iso = P.bc_mode == SHD_BC_ISO ? P.bc[g] : 0.f;
    const bool bc_full = P.bc_mode == SHD_BC_FULL;
    const int tid = threadIdx.x;
    // the CTA holding the row one step upwind of this CTA's boundary row
    const int pr = o.s1 > 0 ? r - 1 : (o.s1 < 0 ? r + 1 : -1);
    const bool has_peer = pr >= 0 && pr < C;
    float4 *Qpeer = has_peer ? cl.map_shared_rank(Q, pr) : Q;
    const int jpeer = has_peer ? pr * R * n2 : 0;  // first node of the peer's block

    // bit u of `face`: node j0 + tid + NT u is on an inflow face of an
    // in-plane axis; bit u of `halo`: its row-upwind neighbours are the peer's
    unsigned face = 0, halo = 0;
    {
        const int first1 = o.s1 > 0 ? 0 : n1 - 1, first2 = o.s2 > 0 ? 0 : n2 - 1;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int jl = tid + NT * u;
            if (jl >= nloc) break;
            const int i1 = (j0 + jl) / n2, i2 = (j0 + jl) - i1 * n2;
            if ((o.s1 != 0 && i1 == first1) || (o.s2 != 0 && i2 == first2)) face |= 1u << u;
            const int jn = jl - o.s1 * n2;
            if (jn < 0 || jn >= nloc) halo |= 1u << u;
        }
    }
    const int d1 = o.s1 * n2, d2 = o.s2;
    // moving-node bits of this thread's chi pieces, as in k_sweep_pp
    constexpr int MP = (U + 3) / 4;
    unsigned long long mw[MP];
    int mwin = -1;

    auto issue = [&](int step) {
        if (step < nd) {
            const int id = o.sd > 0 ? step : nd - 1 - step;
            const long long pb = base + (long long)id * plane + j0;
            float *rg = ring + (size_t)(step & 1) * 3 * pstride;
            const int nv = nloc / 4;  // 16-byte pieces per array
            for (int q = tid; q < nv; q += NT) cp_async_n<16>(&rg[q * 4], &I[pb + q * 4]);
            for (int q = tid; q < nv; q += NT) cp_async_n<16>(&rg[pstride + q * 4], &eta[pb + q * 4]);
            if (CB && (id >> 6) != mwin) {
                mwin = id >> 6;
#pragma unroll
                for (int pi = 0; pi < MP; ++pi) {
                    const int q = tid + pi * NT;
                    mw[pi] = q < nv ? mb[(size_t)mwin * npc + (j0 >> 2) + q] : 0ull;
                }
            }
#pragma unroll
            for (int pi = 0; pi < MP; ++pi) {
                const int q = tid + pi * NT;
                if (q >= nv) break;
                const int off = q * 4;
                const float *src = chi + pb + off;
                if (CB && !((mw[pi] >> (id & 63)) & 1ull)) src = c0base + (long long)id * plane + j0 + off;
                cp_async_n<16>(&rg[2 * pstride + off], src);
            }
        }
        asm volatile("cp.async.commit_group;\n" ::);
    };

    // The cluster barrier is split: a thread arrives (release: its writes of
    // the plane buffer and its landed copies) and then stores the previous
    // plane's intensities to global memory before it waits, so that a release
    // never waits for that plane's global stores; the next arrival covers
    // them a plane later.
    float inew_u[U];
    long long pb_prev = -1;
    auto store_prev = [&]() {
        if (pb_prev < 0) return;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = tid + NT * u;
            if (j >= nloc) break;
            I[pb_prev + j] = inew_u[u];
        }
    };
    issue(0);
    for (int step = 0; step < nd; ++step) {
        asm volatile("cp.async.wait_group 0;\n" ::);
        // this plane's copies and the cluster's previous-plane state are visible after the wait
        asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
        store_prev();
        asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");
        issue(step + 1);
        const float *rg = ring + (size_t)(step & 1) * 3 * pstride;
        const size_t pprev = (size_t)((step + 1) & 1) * pstride;
        const float4 *Qp = Q + pprev;                   // plane step - 1, this CTA's rows
        const float4 *Qr = Qpeer + pprev;               // plane step - 1, the peer's rows
        float4 *Qn = Q + (size_t)(step & 1) * pstride;  // plane step
        const bool first = step == 0;
        const int id = o.sd > 0 ? step : nd - 1 - step;
        const long long pb = base + (long long)id * plane + j0;
        pb_prev = pb;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = tid + NT * u;
            if (j >= nloc) break;
            const float In = rg[j];
            const float ct = rg[2 * pstride + j] + kap;
            const float st = ct > 0.f ? (rg[pstride + j] + kap * In) * hw_rcp(ct) : 0.f;
            float inew;
            if (first || ((face >> u) & 1u)) {
                inew = bc_full ? P.bc[pb + j] : bc_iso;
            } else {
                const float4 q00 = Qp[j], q01 = Qp[j - d2];
                float4 q10, q11;
                if ((halo >> u) & 1u) {
                    const int jr = j0 + j - d1 - jpeer;  // the peer's local index
                    q10 = Qr[jr];
                    q11 = Qr[jr - d2];
                } else {
                    q10 = Qp[j - d1];
                    q11 = Qp[j - d1 - d2];
                }
                const float iu = w00 * q00.x + w10 * q10.x + w01 * q01.x + w11 * q11.x;
                const float su = w00 * q00.y + w10 * q10.y + w01 * q01.y + w11 * q11.y;
                const float cu = w00 * q00.z + w10 * q10.z + w01 * q01.z + w11 * q11.z;
                const float dtau = s * 0.5f * (cu + ct);
                float ew, wp, wu;
                if constexpr (WIDE) sc_weights<float>(dtau, ew, wp, wu);
                else sc_weights_narrow_x2(dtau, ew, wp, wu);
                inew = iu * ew + st * wp + su * wu;
            }
            Qn[j] = make_float4(inew, st, ct, 0.f);
            inew_u[u] = inew;
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    asm volatile("barrier.cluster.arrive.release.aligned;\n" ::: "memory");
    store_prev();  // the last plane
    asm volatile("barrier.cluster.wait.acquire.aligned;\n" ::: "memory");  // the peers' reads of this CTA's buffers are done
}

// -------------------------------------------------------------------------
// a4 with the cubic Bezier short characteristic (Sec. 2), any precision, one
// 1024-thread CTA per (ordinate, group).  Besides the upwind point U the
// source's end derivatives need the downwind point D = P + s n on the next
// plane, so the walk runs one plane behind its inputs: iteration t forms
// S~, chi~ of plane t+1 (buffer NX) and sweeps plane t-1, whose downwind
// values (plane t) were formed in iteration t-1.  Plane t-1 writes (I, S~,
// chi~, dS/dtau) of each node into buffer Q for the next plane's upwind
// interpolation.  One barrier per iteration orders both two-slot buffers.
// The end derivative at P is Fritsch-Butland's from the upwind and downwind
// slopes (the upwind slope where D leaves the grid); at U the bilinear mix of
// the upwind face nodes' derivatives over those that have one (the segment's
// slope if none); at inflow nodes the downwind slope, none (NaN) without D.
// Control points a third of the segment along them, clamped into [S_U, S_P].
// -------------------------------------------------------------------------
template <class T>
struct alignas(4 * sizeof(T)) Quad4 {
    T x, y, z, w;
};
template <class T>
struct alignas(2 * sizeof(T)) Pair2 {
    T x, y;
};

template <class T>
__device__ inline T clamp_between(T v, T a, T b)
{
    const T lo = a < b ? a : b, hi = a < b ? b : a;
    return v < lo ? lo : (v > hi ? hi : v);
}

template <class T, int U, bool WIDE>
__global__ void __launch_bounds__(1024, 1) k_sweep_bez(Prob<T> P, T *__restrict__ I, const T *__restrict__ eta,
                                                       const T *__restrict__ chi, int pstride)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    constexpr int NT = 1024;
    const int k = blockIdx.x / P.G;
    const int g = blockIdx.x - k * P.G;
    const Ordinate o = P.ord[k];
    const int dims[3] = {P.nx, P.ny, P.nz};
    const int nd = dims[o.d], n1 = dims[o.e1], n2 = dims[o.e2];
    const int plane = n1 * n2;
    Quad4<T> *Q = reinterpret_cast<Quad4<T> *>(smem_raw);         // [2][pstride]
    Pair2<T> *NX = reinterpret_cast<Pair2<T> *>(Q + 2 * (size_t)pstride);  // [2][pstride]
    const long long base = ((long long)k * P.G + g) * P.Nc;
    const T fr1 = (T)o.fr1, fr2 = (T)o.fr2, s = (T)o.s, kap = P.kappa;
    const T w00 = (T(1) - fr1) * (T(1) - fr2), w10 = fr1 * (T(1) - fr2), w01 = (T(1) - fr1) * fr2, w11 = fr1 * fr2;
    const T bc_iso = P.bc_mode == SHD_BC_ISO ? P.bc[g] : T(0);
    const bool bc_full = P.bc_mode == SHD_BC_FULL;
    const int tid = threadIdx.x;
    // bit u of fin / fout: node tid + NT u is on an inflow / outflow face of
    // an in-plane axis (no upwind / no downwind point inside the grid)
    unsigned fin = 0, fout = 0;
    {
        const int first1 = o.s1 > 0 ? 0 : n1 - 1, first2 = o.s2 > 0 ? 0 : n2 - 1;
        const int last1 = o.s1 > 0 ? n1 - 1 : 0, last2 = o.s2 > 0 ? n2 - 1 : 0;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = tid + NT * u;
            const int i1 = j / n2, i2 = j - i1 * n2;
            if ((o.s1 != 0 && i1 == first1) || (o.s2 != 0 && i2 == first2)) fin |= 1u << u;
            if ((o.s1 != 0 && i1 == last1) || (o.s2 != 0 && i2 == last2)) fout |= 1u << u;
        }
    }
    const int d1 = o.s1 * n2, d2 = o.s2;
    auto plane_id = [&](int step) { return o.sd > 0 ? step : nd - 1 - step; };
    auto form = [&](int step, const T *In, const T *Et, const T *Ch) {
        Pair2<T> *dst = NX + (size_t)(step & 1) * pstride;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = tid + NT * u;
            if (j >= plane) break;
            const T ct = Ch[u] + kap;
            Pair2<T> v;
            v.x = ct > T(0) ? (Et[u] + kap * In[u]) / ct : T(0);
            v.y = ct;
            dst[j] = v;
        }
    };
    {
        T In[U], Et[U], Ch[U];
        const long long pb = base + (long long)plane_id(0) * plane;
#pragma unroll
        for (int u = 0; u < U; ++u) {
            const int j = tid + NT * u;
            In[u] = Et[u] = Ch[u] = T(0);
            if (j < plane) { In[u] = I[pb + j]; Et[u] = eta[pb + j]; Ch[u] = chi[pb + j]; }
        }
        form(0, In, Et, Ch);
    }
    for (int t = 0; t <= nd; ++t) {
        __syncthreads();
        T In[U], Et[U], Ch[U];
        const bool more = t + 1 < nd;
        if (more) {
            const long long pb = base + (long long)plane_id(t + 1) * plane;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = tid + NT * u;
                In[u] = Et[u] = Ch[u] = T(0);
                if (j < plane) { In[u] = I[pb + j]; Et[u] = eta[pb + j]; Ch[u] = chi[pb + j]; }
            }
        }
        if (t >= 1) {
            const int p = t - 1;
            const long long pb = base + (long long)plane_id(p) * plane;
            const Pair2<T> *own = NX + (size_t)(p & 1) * pstride;
            const Pair2<T> *dn = NX + (size_t)(t & 1) * pstride;
            const Quad4<T> *up = Q + (size_t)(t & 1) * pstride;  // plane p - 1
            Quad4<T> *out = Q + (size_t)(p & 1) * pstride;
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const int j = tid + NT * u;
                if (j >= plane) break;
                const Pair2<T> me = own[j];
                const T sP = me.x, cP = me.y;
                const bool has_d = t < nd && !((fout >> u) & 1u);
                T sD = T(0), cD = T(0);
                if (has_d) {
                    const Pair2<T> a = dn[j], b = dn[j + d1], c2 = dn[j + d2], dd = dn[j + d1 + d2];
                    sD = w00 * a.x + w10 * b.x + w01 * c2.x + w11 * dd.x;
                    cD = w00 * a.y + w10 * b.y + w01 * c2.y + w11 * dd.y;
                }
                const T xd = s * T(0.5) * (cP + cD);
                T inew, dP;
                if (p == 0 || ((fin >> u) & 1u)) {
                    inew = bc_full ? P.bc[pb + j] : bc_iso;
                    // the downwind slope; no derivative (NaN) without a downwind point
                    dP = has_d ? (xd > T(0) ? (sD - sP) / xd : T(0)) : T(NAN);
                } else {
                    const Quad4<T> q00 = up[j], q10 = up[j - d1], q01 = up[j - d2], q11 = up[j - d1 - d2];
                    const T iu = w00 * q00.x + w10 * q10.x + w01 * q01.x + w11 * q11.x;
                    const T su = w00 * q00.y + w10 * q10.y + w01 * q01.y + w11 * q11.y;
                    const T cu = w00 * q00.z + w10 * q10.z + w01 * q01.z + w11 * q11.z;
                    // the upwind face nodes' derivatives, over those that have one
                    T dsum = T(0), dw = T(0);
                    if (!isnan(q00.w)) { dsum += w00 * q00.w; dw += w00; }
                    if (!isnan(q10.w)) { dsum += w10 * q10.w; dw += w10; }
                    if (!isnan(q01.w)) { dsum += w01 * q01.w; dw += w01; }
                    if (!isnan(q11.w)) { dsum += w11 * q11.w; dw += w11; }
                    const T x = s * T(0.5) * (cu + cP);
                    const T slope = x > T(0) ? (sP - su) / x : T(0);
                    const T du = dw > T(0) ? dsum / dw : slope;
                    dP = slope;
                    if (has_d) dP = (x > T(0) && xd > T(0)) ? fb_derivative<T>(slope, (sD - sP) / xd, x, xd) : T(0);
                    const T Cu = clamp_between<T>(su + x * du / T(3), su, sP);
                    const T Cp = clamp_between<T>(sP - x * dP / T(3), su, sP);
                    T e, wU, wCU, wCP, wP;
                    if (WIDE && sizeof(T) == 4 && x > T(kFp64Tau)) {
                        double ed, a1, a2, a3, a4;
                        bezier_weights<double>((double)x, ed, a1, a2, a3, a4);
                        e = (T)ed; wU = (T)a1; wCU = (T)a2; wCP = (T)a3; wP = (T)a4;
                    } else {
                        bezier_weights<T>(x, e, wU, wCU, wCP, wP);
                    }
                    inew = iu * e + wU * su + wCU * Cu + wCP * Cp + wP * sP;
                }
                Quad4<T> v;
                v.x = inew; v.y = sP; v.z = cP; v.w = dP;
                out[j] = v;
                I[pb + j] = inew;
            }
        }
        if (more) form(t + 1, In, Et, Ch);
    }
}

// -------------------------------------------------------------------------
// a5: FP64 diagnostics; pass 1 per-block partials, pass 2 a single block
// adds them in a fixed order (deterministic).
// -------------------------------------------------------------------------
template <class T>
__global__ void k_sums_partial(Prob<T> P, const T *__restrict__ mom, const T *__restrict__ Sp,
                               const T *__restrict__ Sprev, int have_prev, double *partial)
{
    __shared__ double red[4][256];
    double e = 0, ph = 0, num = 0, den = 0;
    const long long nJ = P.Nc * P.G;
    const long long nS = nJ * P.NLM;
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < nJ; i += stride) {
        int g = (int)(i % P.G);
        double J = (double)mom[i * 10];
        double de = P.edges[g + 1] - P.edges[g];
        e += 4.0 * kPi * J * de;
        ph += 4.0 * kPi * J * de / P.centre[g];
    }
    // |S|^2 and |S - S_prev|^2 in working precision over runs of 64 of a
    // thread's elements, each run's sums then added in FP64 (an FP64
    // operation per element would occupy the narrow FP64 pipe)
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    while (i < nS) {
        T dn = T(0), nm = T(0);
        for (int r = 0; r < 64 && i < nS; ++r, i += stride) {
            const T sv = Sp[i];
            dn += sv * sv;
            if (have_prev) {
                const T d = sv - Sprev[i];
                nm += d * d;
            }
        }
        den += (double)dn;
        num += (double)nm;
    }
    red[0][threadIdx.x] = e;
    red[1][threadIdx.x] = ph;
    red[2][threadIdx.x] = num;
    red[3][threadIdx.x] = den;
    __syncthreads();
    for (int w = blockDim.x / 2; w > 0; w >>= 1) {
        if (threadIdx.x < w)
            for (int q = 0; q < 4; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 4) partial[blockIdx.x * 4 + threadIdx.x] = red[threadIdx.x][0];
}

// One CTA of kSumsThreads: thread t adds partials t, t + kSumsThreads, ...
// in order, then a halving tree adds the threads' sums (a fixed order, so
// the result does not change from run to run).
constexpr int kSumsThreads = 256;
__global__ void __launch_bounds__(kSumsThreads) k_sums_final(const double *partial, int nblocks, int have_prev,
                                                             double *out)
{
    __shared__ double red[4][kSumsThreads];
    const int t = threadIdx.x;
    double acc[4] = {0, 0, 0, 0};
    for (int b = t; b < nblocks; b += kSumsThreads)
        for (int q = 0; q < 4; ++q) acc[q] += partial[b * 4 + q];
    for (int q = 0; q < 4; ++q) red[q][t] = acc[q];
    __syncthreads();
    for (int w = kSumsThreads / 2; w > 0; w >>= 1) {
        if (t < w)
            for (int q = 0; q < 4; ++q) red[q][t] += red[q][t + w];
        __syncthreads();
    }
    if (t == 0) {
        out[0] = red[0][0];
        out[1] = red[1][0];
        out[2] = (have_prev && red[3][0] > 0) ? sqrt(red[2][0] / red[3][0]) : 0.0;
    }
}

// -------------------------------------------------------------------------
// Ng acceleration of the Lambda iteration (Sec. 2, the acceleration cited
// there, Ng 1974): from the last four source iterates x0 = S^n, x1 = S^{n-1},
// x2 = S^{n-2}, x3 = S^{n-3} (all (c, g, p) values), the five FP64 inner
// products <Q1,Q1>, <Q1,Q2>, <Q2,Q2>, <Q1,Q3>, <Q2,Q3> of
//   Q1 = x0 - 2 x1 + x2,  Q2 = x0 - x1 - x2 + x3,  Q3 = x0 - x1,
// per CTA (fixed-order tree), then one CTA adds the CTAs' sums in order.
// -------------------------------------------------------------------------
constexpr int kNgThreads = 256;

template <class T>
__global__ void __launch_bounds__(kNgThreads) k_ng_dots(const T *__restrict__ x0, const T *__restrict__ x1,
                                                        const T *__restrict__ x2, const T *__restrict__ x3,
                                                        long long n, double *part)
{
    __shared__ double red[5][kNgThreads];
    double a[5] = {0, 0, 0, 0, 0};
    const long long stride = (long long)gridDim.x * blockDim.x;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += stride) {
        const double v0 = (double)x0[i], v1 = (double)x1[i], v2 = (double)x2[i], v3 = (double)x3[i];
        const double q1 = v0 - 2.0 * v1 + v2, q2 = v0 - v1 - v2 + v3, q3 = v0 - v1;
        a[0] += q1 * q1;
        a[1] += q1 * q2;
        a[2] += q2 * q2;
        a[3] += q1 * q3;
        a[4] += q2 * q3;
    }
    for (int q = 0; q < 5; ++q) red[q][threadIdx.x] = a[q];
    __syncthreads();
    for (int w = kNgThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) part[blockIdx.x * 5 + threadIdx.x] = red[threadIdx.x][0];
}

__global__ void __launch_bounds__(kNgThreads) k_ng_final(const double *part, int nblk, double *out)
{
    __shared__ double red[5][kNgThreads];
    double a[5] = {0, 0, 0, 0, 0};
    for (int b = threadIdx.x; b < nblk; b += kNgThreads)
        for (int q = 0; q < 5; ++q) a[q] += part[b * 5 + q];
    for (int q = 0; q < 5; ++q) red[q][threadIdx.x] = a[q];
    __syncthreads();
    for (int w = kNgThreads / 2; w > 0; w >>= 1) {
        if ((int)threadIdx.x < w)
            for (int q = 0; q < 5; ++q) red[q][threadIdx.x] += red[q][threadIdx.x + w];
        __syncthreads();
    }
    if (threadIdx.x < 5) out[threadIdx.x] = red[threadIdx.x][0];
}

// The extrapolated iterate x0 <- (1 - a - b) x0 + a x1 + b x2 (in FP64).
template <class T>
__global__ void k_ng_combine(T *__restrict__ x0, const T *__restrict__ x1, const T *__restrict__ x2, long long n,
                             double a, double b)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    x0[i] = (T)((1.0 - a - b) * (double)x0[i] + a * (double)x1[i] + b * (double)x2[i]);
}

// -------------------------------------------------------------------------
// Runge-Kutta sub-stepping of a time step (App. A, eq:rk4th).  A holds
// I(t), B the input of the sub-solve just run, I its result; with
// dI = I - B:  acc = dI (first) or acc + dI;  then either the next input
// I = B = A + c dI, or (last) the new state I = A + acc.
// -------------------------------------------------------------------------
template <class T>
__global__ void k_rk_stage(T *__restrict__ I, const T *__restrict__ A, T *__restrict__ B, T *__restrict__ acc,
                           long long n, T cnext, int first, int last)
{
    const long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i >= n) return;
    const T d = I[i] - B[i];
    const T s = first ? d : acc[i] + d;
    if (last) {
        I[i] = A[i] + s;
        return;
    }
    acc[i] = s;
    const T x = A[i] + cnext * d;
    I[i] = x;
    B[i] = x;
}

// -------------------------------------------------------------------------
// Compton scattering off thermal electrons (the temperature field's reading
// of Sec. 2.3): the kernel of a photon of energy eps (incident group g')
// scattered through the laboratory cosine mu into group g, averaged over
// isotropic Maxwell-Juttner electrons at temperature theta:
//   K_l[g][g'] = (2 pi / de_g) Int_g' d eps Int d mu P_l(mu)
//                < (dsigma/dOmega1)_e (eps1/eps) 1[eps1 in g] >_theta
// with eps' = gamma eps (1 - beta mu_e), eps1 = eps (1 - beta mu_e) /
// ((1 - beta mu_e1) + (eps/gamma)(1 - mu)), eps1' = gamma eps1 (1 - beta
// mu_e1), 1 - cos T' = 1/eps1' - 1/eps', and (dsigma/dOmega1)_e = (1 - beta
// mu_e) (3/16 pi) (eps1/eps')^2 (eps'/eps1' + eps1'/eps' - sin^2 T');
// sigma_out[g'] = (1/de_g') Int_g' d eps <(1 - beta mu_e) sigma_KN(eps')>.
// Product quadrature (FP64): TN_E points in ln(eps), TN_MU in mu, and over
// the electrons TN_S in s = sqrt((gamma - 1)/theta) on [0, sqrt 40] (density
// gamma^2 beta e^(-s^2) 2 theta s, normalised on the rule), TN_ME in their
// direction cosine, TN_PHI azimuths at midpoints.  One CTA per (g', theta_i);
// shared-memory atomics collect the contributions of every final group.
// -------------------------------------------------------------------------
constexpr int TN_E = 16, TN_MU = 48, TN_S = 24, TN_ME = 16, TN_PHI = 16;
constexpr double TN_SMAX = 6.324555320336759;  // sqrt(40)

__device__ inline double sigma_kn_total(double x)
{
    if (x < 1e-4) return 1.0 - 2.0 * x + 5.2 * x * x;
    const double l = log1p(2.0 * x);
    return 0.75 * ((1.0 + x) / (x * x * x) * (2.0 * x * (1.0 + x) / (1.0 + 2.0 * x) - l) + l / (2.0 * x) -
                   (1.0 + 3.0 * x) / ((1.0 + 2.0 * x) * (1.0 + 2.0 * x)));
}

__global__ void __launch_bounds__(256) k_kn_thermal_table(int G, const double *__restrict__ edges, int L,
                                                          const double *__restrict__ quad, double *Kth, double *soth)
{
    extern __shared__ double tsm[];
    double *acc = tsm;                         // [L+1][G]
    double *gam = acc + (size_t)(L + 1) * G;  // [TN_S]
    double *bet = gam + TN_S;
    double *wel = bet + TN_S;
    double *tot = wel + TN_S;                 // [1]
    const double *xs = quad, *ws = xs + TN_S, *xme = ws + TN_S, *wme = xme + TN_ME, *xmu = wme + TN_ME,
                 *wmu = xmu + TN_MU, *xe = wmu + TN_MU, *we = xe + TN_E;
    const int gp = blockIdx.x % G, it = blockIdx.x / G;
    const double theta = pow(10.0, kThermalLg0 + it * kThermalDlg);
    for (int i = threadIdx.x; i < (L + 1) * G; i += blockDim.x) acc[i] = 0.0;
    if (threadIdx.x < TN_S) {
        const int i = threadIdx.x;
        const double sv = 0.5 * TN_SMAX * (xs[i] + 1.0);
        gam[i] = 1.0 + theta * sv * sv;
        bet[i] = sqrt(1.0 - 1.0 / (gam[i] * gam[i]));
        wel[i] = 0.5 * TN_SMAX * ws[i] * gam[i] * gam[i] * bet[i] * exp(-sv * sv) * 2.0 * theta * sv;
    }
    if (threadIdx.x == 0) *tot = 0.0;
    __syncthreads();
    if (threadIdx.x == 0) {
        double sum = 0.0;
        for (int i = 0; i < TN_S; ++i) sum += wel[i];
        for (int i = 0; i < TN_S; ++i) wel[i] /= sum;
    }
    __syncthreads();
    const double t0 = log(edges[gp]), t1 = log(edges[gp + 1]);
    const double ht = 0.5 * (t1 - t0), mt = 0.5 * (t1 + t0);
    // the out-scattering cross-section: (eps, electron speed) pairs per thread
    for (int q = threadIdx.x; q < TN_E * TN_S; q += blockDim.x) {
        const int ie = q / TN_S, is = q - ie * TN_S;
        const double eps = exp(mt + ht * xe[ie]);
        const double weps = we[ie] * ht * eps;
        double a = 0.0;
        for (int im = 0; im < TN_ME; ++im) {
            const double f = 1.0 - bet[is] * xme[im];
            a += 0.5 * wme[im] * f * sigma_kn_total(gam[is] * eps * f);
        }
        atomicAdd(tot, weps * wel[is] * a);
    }
    // the kernel: (eps, mu) pairs per thread, the electrons in a loop
    double pl[16];
    for (int q = threadIdx.x; q < TN_E * TN_MU; q += blockDim.x) {
        const int ie = q / TN_MU, iu = q - ie * TN_MU;
        const double eps = exp(mt + ht * xe[ie]);
        const double weps = we[ie] * ht * eps;
        const double mu = xmu[iu], smu = sqrt(1.0 - mu * mu);
        pl[0] = 1.0;
        if (L >= 1) pl[1] = mu;
        for (int l = 2; l <= L; ++l) pl[l] = ((2.0 * l - 1.0) * mu * pl[l - 1] - (l - 1.0) * pl[l - 2]) / l;
        for (int is = 0; is < TN_S; ++is) {
            const double b = bet[is], gm = gam[is];
            for (int im = 0; im < TN_ME; ++im) {
                const double cme = xme[im], sme = sqrt(1.0 - cme * cme);
                const double a = 1.0 - b * cme;
                for (int ip = 0; ip < TN_PHI; ++ip) {
                    const double phe = 2.0 * kPi * (ip + 0.5) / TN_PHI;
                    const double mue1 = sme * cos(phe) * smu + cme * mu;
                    const double eps1 = eps * a / ((1.0 - b * mue1) + (eps / gm) * (1.0 - mu));
                    if (!(eps1 >= edges[0] && eps1 < edges[G])) continue;
                    int lo = 0, hi = G - 1;  // the group holding eps1
                    while (lo < hi) {
                        const int mid = (lo + hi + 1) >> 1;
                        if (edges[mid] <= eps1) lo = mid;
                        else hi = mid - 1;
                    }
                    const double ep = gm * eps * a, e1p = gm * eps1 * (1.0 - b * mue1);
                    const double ct = 1.0 - (1.0 / e1p - 1.0 / ep);
                    const double r = eps1 / ep;
                    double dsdo = a * 3.0 / (16.0 * kPi) * r * r * (ep / e1p + e1p / ep - (1.0 - ct * ct));
                    dsdo *= eps1 / eps;
                    const double wgt = weps * wmu[iu] * wel[is] * 0.5 * wme[im] / TN_PHI * dsdo;
                    for (int l = 0; l <= L; ++l) atomicAdd(&acc[l * G + lo], wgt * pl[l]);
                }
            }
        }
    }
    __syncthreads();
    const size_t per = (size_t)(L + 1) * G * G;
    for (int i = threadIdx.x; i < (L + 1) * G; i += blockDim.x) {
        const int l = i / G, g = i - l * G;
        Kth[(size_t)it * per + ((size_t)l * G + g) * G + gp] = 2.0 * kPi * acc[i] / (edges[g + 1] - edges[g]);
    }
    if (threadIdx.x == 0) soth[(size_t)it * G + gp] = *tot / (edges[gp + 1] - edges[gp]);
}

// -------------------------------------------------------------------------
// The thermal form of k_source_kn (FP32): chunks of nodes of one temperature
// bracket b, the CTA persistent over chunks; per chunk the transposed K of
// tables b and b+1 in shared memory, tiles of TN of the chunk's nodes (each
// node's I_lm row contiguous) through the two-stage ring, and per unit two
// accumulator sets, blended by the node's weight w of the upper table:
// S_p = n_e/chi0 ((1 - w) sum_g' K_b I + w sum_g' K_(b+1) I) + delta_p0
// sqrt(4 pi) eta0/chi0.
// -------------------------------------------------------------------------
template <int TN>
__global__ void __launch_bounds__(512, 1) k_source_kn_th(Prob<float> P, const float *__restrict__ Ip,
                                                         float *__restrict__ Sp, const float *__restrict__ mom,
                                                         const float *__restrict__ Sprev, int have_prev,
                                                         double *partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][16];
    __shared__ long long sC[2][TN];
    const int G = P.G, NLM = P.NLM, L = P.L;
    const int Gb = (G + 3) / 4, G4 = 4 * Gb;
    const int row_f = G * NLM, tile_f = TN * row_f;
    const size_t kper = (size_t)(L + 1) * G * G4;
    float *sKa = reinterpret_cast<float *>(smem_raw);  // [L+1][G][G4] transposed, table b
    float *sKb = sKa + kper;                            // table b + 1
    float *sI = sKb + kper;                             // [2][TN][G][NLM]
    float *sR = sI + (size_t)2 * tile_f;                // [TN][G4]
    float *sE = sR + TN * G4;                           // [TN][G4]
    float *sW = sE + TN * G4;                           // [TN]
    const int tid = threadIdx.x, nt = blockDim.x;
    const int nunit = Gb * NLM;
    double e = 0, ph = 0, num = 0, den = 0;
    for (int ch = blockIdx.x; ch < P.nthchunk; ch += gridDim.x) {
        const int4 cd = P.thchunk[ch];
        const int ntile = (cd.y + TN - 1) / TN;
        asm volatile("cp.async.wait_group 0;\n" ::);
        __syncthreads();  // the previous chunk's reads of the tables and buffers are done
        const size_t per = (size_t)(L + 1) * G * G;
        for (int i = tid; i < (int)kper; i += nt) {
            const int l = i / (G * G4), rem = i - l * G * G4, gp = rem / G4, g = rem - gp * G4;
            const size_t src = ((size_t)l * G + g) * G + gp;
            sKa[i] = g < G ? P.thK[(size_t)cd.z * per + src] : 0.f;
            sKb[i] = g < G ? P.thK[(size_t)(cd.z + 1) * per + src] : 0.f;
        }
        auto load = [&](int t, int buf) {
            if (t < ntile) {
                const int j0 = t * TN, nn = cd.y - j0 < TN ? cd.y - j0 : TN;
                const int pr = row_f / 4;  // 16-byte pieces of a node's row
                for (int q = tid; q < nn * pr; q += nt) {
                    const int n = q / pr, qq = q - n * pr;
                    const long long c = P.thperm[cd.x + j0 + n];
                    cp_async_n<16>(sI + (size_t)buf * tile_f + (size_t)n * row_f + 4 * qq, Ip + c * row_f + 4 * qq);
                }
                if (tid < nn) sC[buf][tid] = P.thperm[cd.x + j0 + tid];
            }
            asm volatile("cp.async.commit_group;\n" ::);
        };
        load(0, 0);
        for (int t = 0; t < ntile; ++t) {
            const int buf = t & 1;
            const int nn = cd.y - t * TN < TN ? cd.y - t * TN : TN;
            asm volatile("cp.async.wait_group 0;\n" ::);
            __syncthreads();  // the tile (and at t = 0 the tables) landed; the previous tile is done
            load(t + 1, buf ^ 1);
            for (int i = tid; i < TN * G4; i += nt) {
                const int n = i / G4, g = i - n * G4;
                float r = 0.f, em = 0.f;
                if (n < nn && g < G) {
                    const long long c = sC[buf][n];
                    const float chi = P.chi0[c * G + g];
                    if (chi > 0.f) {
                        r = P.ne[c] / chi;
                        em = 3.5449077018110320546f * P.emis0[c * G + g] / chi;  // sqrt(4 pi)
                    }
                }
                sR[i] = r;
                sE[i] = em;
            }
            if (tid < TN) sW[tid] = tid < nn ? P.thw[sC[buf][tid]] : 0.f;
            for (int i = tid; i < nn * G; i += nt) {
                const int n = i / G, g = i - n * G;
                const double J = (double)mom[(sC[buf][n] * G + g) * 10];
                const double de = P.edges[g + 1] - P.edges[g];
                e += 4.0 * kPi * J * de;
                ph += 4.0 * kPi * J * de / P.centre[g];
            }
            __syncthreads();
            const float *tI = sI + (size_t)buf * tile_f;
            for (int u = tid; u < nunit; u += nt) {
                int l = (int)sqrtf((float)(u / Gb));
                while (Gb * (l + 1) * (l + 1) <= u) ++l;
                while (Gb * l * l > u) --l;
                const int r = u - Gb * l * l, gb = r / (2 * l + 1), p = l * l + (r - gb * (2 * l + 1));
                float aa[4][TN], ab[4][TN];
#pragma unroll
                for (int j = 0; j < 4; ++j)
#pragma unroll
                    for (int n = 0; n < TN; ++n) aa[j][n] = ab[j][n] = 0.f;
                const float4 *ka = reinterpret_cast<const float4 *>(sKa + (size_t)l * G * G4) + gb;
                const float4 *kb = reinterpret_cast<const float4 *>(sKb + (size_t)l * G * G4) + gb;
                const float *ir = tI + p;
#pragma unroll 2
                for (int gp = 0; gp < G; ++gp) {
                    const float4 a4 = ka[(size_t)gp * Gb], b4 = kb[(size_t)gp * Gb];
                    float iv[TN];
#pragma unroll
                    for (int n = 0; n < TN; ++n) iv[n] = ir[((size_t)n * G + gp) * NLM];
#pragma unroll
                    for (int n = 0; n < TN; ++n) {
                        aa[0][n] += a4.x * iv[n]; aa[1][n] += a4.y * iv[n];
                        aa[2][n] += a4.z * iv[n]; aa[3][n] += a4.w * iv[n];
                        ab[0][n] += b4.x * iv[n]; ab[1][n] += b4.y * iv[n];
                        ab[2][n] += b4.z * iv[n]; ab[3][n] += b4.w * iv[n];
                    }
                }
                float dn = 0.f, nmr = 0.f;
#pragma unroll
                for (int j = 0; j < 4; ++j) {
                    const int g = 4 * gb + j;
                    const bool gv = g < G;
                    float sv[TN], pv[TN];
                    long long o[TN];
#pragma unroll
                    for (int n = 0; n < TN; ++n) {
                        const float w = sW[n];
                        sv[n] = sR[n * G4 + g] * ((1.f - w) * aa[j][n] + w * ab[j][n]);
                        if (p == 0) sv[n] += sE[n * G4 + g];
                        o[n] = (sC[buf][n] * G + g) * NLM + p;
                        pv[n] = 0.f;
                    }
                    if (have_prev) {
#pragma unroll
                        for (int n = 0; n < TN; ++n)
                            if (gv && n < nn) pv[n] = Sprev[o[n]];
                    }
#pragma unroll
                    for (int n = 0; n < TN; ++n) {
                        if (gv && n < nn) {
                            Sp[o[n]] = sv[n];
                            dn += sv[n] * sv[n];
                            const float d = sv[n] - pv[n];
                            if (have_prev) nmr += d * d;
                        }
                    }
                }
                den += (double)dn;
                num += (double)nmr;
            }
        }
    }
    asm volatile("cp.async.wait_group 0;\n" ::);
    const int warp = tid >> 5, lane = tid & 31, nw = nt >> 5;
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, o);
        ph += __shfl_down_sync(0xffffffffu, ph, o);
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if (lane == 0) {
        red[0][warp] = e;
        red[1][warp] = ph;
        red[2][warp] = num;
        red[3][warp] = den;
    }
    __syncthreads();
    if (tid < 4) {
        double a = 0;
        for (int w = 0; w < nw; ++w) a += red[tid][w];
        partial[blockIdx.x * 4 + tid] = a;
    }
}

// -------------------------------------------------------------------------
// a2 (+ a5 partials) with thermal electrons: chunks of nodes of one
// temperature bracket b; the CTA holds K of tables b and b+1, each warp
// stages a node's I_lm and forms S_p = n_e/chi0 ((1 - w) sum_g' K_b I +
// w sum_g' K_(b+1) I) + delta_p0 sqrt(4 pi) eta0/chi0 (w the node's weight
// of the upper table), with the FP64 partial sums of k_source_sums.
// -------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_source_thermal(Prob<T> P, const T *__restrict__ Ip, T *__restrict__ Sp,
                                                        const T *__restrict__ mom, const T *__restrict__ Sprev,
                                                        int have_prev, double *partial)
{
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ double red[4][8];
    const int G = P.G, NLM = P.NLM, L = P.L;
    const int W = blockDim.x >> 5;
    const size_t per = (size_t)(L + 1) * G * G;
    T *Ka = reinterpret_cast<T *>(smem_raw);
    T *Kb = Ka + per;
    T *sI = Kb + per;  // [W][G][NLM]
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    T *wI = sI + (size_t)warp * G * NLM;
    double e = 0, ph = 0, num = 0, den = 0;
    for (int ch = blockIdx.x; ch < P.nthchunk; ch += gridDim.x) {
        const int4 cd = P.thchunk[ch];
        __syncthreads();  // the previous chunk's tables are no longer read
        for (size_t i = threadIdx.x; i < per; i += blockDim.x) {
            Ka[i] = P.thK[(size_t)cd.z * per + i];
            Kb[i] = P.thK[(size_t)(cd.z + 1) * per + i];
        }
        __syncthreads();
        for (int j = warp; j < cd.y; j += W) {
            const long long c = P.thperm[cd.x + j];
            const long long base = c * G * NLM;
            const T ne = P.ne[c], w = P.thw[c];
            for (int i = lane; i < G * NLM; i += 32) wI[i] = Ip[base + i];
            __syncwarp();
            T dn = T(0), nm = T(0);  // the node's residual parts, as in k_source_sums
            for (int p = lane; p < NLM; p += 32) {
                int l = 0;
                while ((l + 1) * (l + 1) <= p) ++l;
                for (int g = 0; g < G; ++g) {
                    const T chi = P.chi0[c * G + g];
                    T s = T(0);
                    if (chi > T(0)) {
                        const T *ra = Ka + (size_t)l * G * G + (size_t)g * G, *rb = Kb + (size_t)l * G * G + (size_t)g * G;
                        T aa = T(0), ab = T(0);
                        for (int gp = 0; gp < G; ++gp) {
                            const T v = wI[gp * NLM + p];
                            aa += ra[gp] * v;
                            ab += rb[gp] * v;
                        }
                        s = ne / chi * ((T(1) - w) * aa + w * ab);
                        if (p == 0) s += T(3.5449077018110320546) * P.emis0[c * G + g] / chi;  // sqrt(4 pi)
                    }
                    const long long i = base + (long long)g * NLM + p;
                    Sp[i] = s;
                    dn += s * s;
                    if (have_prev) {
                        const T d = s - Sprev[i];
                        nm += d * d;
                    }
                }
            }
            den += (double)dn;
            num += (double)nm;
            for (int g = lane; g < G; g += 32) {
                const double J = (double)mom[(c * G + g) * 10];
                const double de = P.edges[g + 1] - P.edges[g];
                e += 4.0 * kPi * J * de;
                ph += 4.0 * kPi * J * de / P.centre[g];
            }
            __syncwarp();
        }
    }
    for (int o = 16; o > 0; o >>= 1) {
        e += __shfl_down_sync(0xffffffffu, e, o);
        ph += __shfl_down_sync(0xffffffffu, ph, o);
        num += __shfl_down_sync(0xffffffffu, num, o);
        den += __shfl_down_sync(0xffffffffu, den, o);
    }
    if (lane == 0) {
        red[0][warp] = e;
        red[1][warp] = ph;
        red[2][warp] = num;
        red[3][warp] = den;
    }
    __syncthreads();
    if (threadIdx.x < 4) {
        double acc = 0;
        for (int w = 0; w < W; ++w) acc += red[threadIdx.x][w];
        partial[blockIdx.x * 4 + threadIdx.x] = acc;
    }
}

// -------------------------------------------------------------------------
// layout conversions
// -------------------------------------------------------------------------
template <class T>
__global__ void k_canon_to_do(Prob<T> P, const double *__restrict__ src, T *__restrict__ dst, long long c0,
                              long long nc)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int G = P.G, N = P.N;
    long long n = nc * G * N;
    if (i >= n) return;
    int k = (int)(i % N);
    long long cg = i / N;
    int g = (int)(cg % G);
    long long c = c0 + cg / G;
    int ix, iy, iz;
    node_xyz(c, P.nx, P.ny, ix, iy, iz);
    const int ki = P.mesh2int[k];  // canonical arrays are in mesh order
    dst[((long long)ki * G + g) * P.Nc + perm_offset(P.ord[ki].d, ix, iy, iz, P.nx, P.ny, P.nz)] = (T)src[i];
}

template <class T>
__global__ void k_do_to_canon(Prob<T> P, const T *__restrict__ src, double *__restrict__ dst, long long c0,
                              long long nc)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    const int G = P.G, N = P.N;
    long long n = nc * G * N;
    if (i >= n) return;
    int k = (int)(i % N);
    long long cg = i / N;
    int g = (int)(cg % G);
    long long c = c0 + cg / G;
    int ix, iy, iz;
    node_xyz(c, P.nx, P.ny, ix, iy, iz);
    const int ki = P.mesh2int[k];  // canonical arrays are in mesh order
    dst[i] = (double)src[((long long)ki * G + g) * P.Nc + perm_offset(P.ord[ki].d, ix, iy, iz, P.nx, P.ny, P.nz)];
}

template <class T>
__global__ void k_convert(const double *__restrict__ src, T *__restrict__ dst, long long n)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (T)src[i];
}

template <class T>
__global__ void k_convert_back(const T *__restrict__ src, double *__restrict__ dst, long long n)
{
    long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x;
    if (i < n) dst[i] = (double)src[i];
}

// -------------------------------------------------------------------------
// Klein-Nishina multigroup table (Sec. 2.3, eq:comptoncross), FP64, one
// thread per (final group g, incident group g'):
//   K_l[g][g'] = (2 pi / de_g) Int_{g'} d eps Int d mu P_l(mu) dsigma/dOmega (eps1/eps) 1[eps1 in g]
//   sigma_out[g'] = (1/de_g') Int_{g'} sigma_KN(eps) d eps        (sigma_T units)
// dsigma/dOmega = (3/16pi) r^2 (1/r + r - sin^2), r = eps1/eps = 1/(1+eps(1-mu)).
// Angles are integrated in ln(eps1) (mu = 1 + 1/eps - 1/eps1), energies in
// ln(eps), each on pieces split where a group edge stops being reachable.
// -------------------------------------------------------------------------
__device__ inline double kn_angle_integral(int l, double eps, double lo, double hi, int weighted,
                                           const double *gx, const double *gw, int nq)
{
    double s0 = log(lo), s1 = log(hi);
    double hs = 0.5 * (s1 - s0), ms = 0.5 * (s1 + s0);
    double acc = 0.0;
    for (int i = 0; i < nq; ++i) {
        double e1 = exp(ms + hs * gx[i]);
        double mu = 1.0 + 1.0 / eps - 1.0 / e1;
        mu = fmin(1.0, fmax(-1.0, mu));
        double r = e1 / eps;
        double dsdo = 3.0 / (16.0 * kPi) * r * r * (1.0 / r + r - (1.0 - mu * mu));
        // Legendre P_l(mu) by recurrence
        double pl = 1.0;
        if (l >= 1) {
            double p0 = 1.0, p1 = mu;
            for (int j = 2; j <= l; ++j) {
                double p2 = ((2.0 * j - 1.0) * mu * p1 - (j - 1.0) * p0) / j;
                p0 = p1;
                p1 = p2;
            }
            pl = p1;
        }
        double f = pl * dsdo / e1;
        if (weighted) f *= r;
        acc += gw[i] * f;
    }
    return acc * hs;
}

__global__ void k_kn_table(int G, const double *edges, int L, double *K, double *sigma_out, const double *gx,
                           const double *gw, int nq)
{
    int idx = blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= G * G) return;
    int g = idx / G, gp = idx - g * G;
    double ea = edges[gp], eb = edges[gp + 1];
    // breakpoints of the incident-energy integral
    double bp[2 * 257 + 2];
    int nb = 0;
    bp[nb++] = ea;
    bp[nb++] = eb;
    for (int j = 0; j <= G; ++j) {
        double e = edges[j];
        if (e > ea && e < eb) bp[nb++] = e;
        if (e < 0.5) {
            double e2 = e / (1.0 - 2.0 * e);
            if (e2 > ea && e2 < eb) bp[nb++] = e2;
        }
    }
    for (int i = 1; i < nb; ++i) {  // insertion sort
        double v = bp[i];
        int j = i - 1;
        while (j >= 0 && bp[j] > v) { bp[j + 1] = bp[j]; --j; }
        bp[j + 1] = v;
    }
    double acc[16];
    for (int l = 0; l <= L; ++l) acc[l] = 0.0;
    double tot = 0.0;
    for (int sgm = 0; sgm + 1 < nb; ++sgm) {
        if (!(bp[sgm + 1] > bp[sgm])) continue;
        double t0 = log(bp[sgm]), t1 = log(bp[sgm + 1]);
        double ht = 0.5 * (t1 - t0), mt = 0.5 * (t1 + t0);
        for (int i = 0; i < nq; ++i) {
            double eps = exp(mt + ht * gx[i]);
            double wq = gw[i] * ht * eps;
            double e1min = eps / (1.0 + 2.0 * eps), e1max = eps;
            if (g == 0) tot += wq * 2.0 * kPi * kn_angle_integral(0, eps, e1min, e1max, 0, gx, gw, nq);
            double lo = fmax(edges[g], e1min), hi = fmin(edges[g + 1], e1max);
            if (!(hi > lo)) continue;
            for (int l = 0; l <= L; ++l) acc[l] += wq * kn_angle_integral(l, eps, lo, hi, 1, gx, gw, nq);
        }
    }
    double norm = 2.0 * kPi / (edges[g + 1] - edges[g]);
    for (int l = 0; l <= L; ++l) K[((size_t)l * G + g) * G + gp] = acc[l] * norm;
    if (g == 0) sigma_out[gp] = tot / (eb - ea);
}

// -------------------------------------------------------------------------
// launchers
// -------------------------------------------------------------------------
static inline unsigned blocks_for(long long n, int bs) { return (unsigned)((n + bs - 1) / bs); }

static int sweep_plane_max(const shd_ctx *c)
{
    int a = c->nx * c->ny, b = c->ny * c->nz, d = c->nx * c->nz;
    int m = a > b ? a : b;
    return m > d ? m : d;
}
size_t sweep_smem_bytes(const shd_ctx *c) { return (size_t)3 * c->esize * sweep_plane_max(c); }

// chi at rest in every ordinate's sweep layout: row (k, g) of chi_lab is row
// (d(k), g) of the chi0 layouts, d(k) the sweep axis of ordinate k.
template <class T>
__global__ void k_chi_rest_fill(Prob<T> P, const T *__restrict__ chi0L, T *__restrict__ chi,
                                const int *__restrict__ dirty, int force)
{
    if (!force && *dirty == 0) return;  // chi0 unchanged since the last fill
    const long long rows = (long long)P.N * P.G;
    for (long long row = blockIdx.y; row < rows; row += gridDim.y) {
        const int k = (int)(row / P.G), g = (int)(row - (long long)k * P.G);
        const T *src = chi0L + ((long long)P.ord[k].d * P.G + g) * P.Nc;
        T *dst = chi + row * P.Nc;
        for (long long o = (long long)blockIdx.x * blockDim.x + threadIdx.x; o < P.Nc;
             o += (long long)gridDim.x * blockDim.x)
            dst[o] = src[o];
    }
}

template <class T>
cudaError_t launch_chi_rest_fill(const shd_ctx *ctx, T *chi, cudaStream_t st, bool force)
{
    if (!ctx->d_chi0L || !ctx->d_chi_dirty) return cudaErrorInvalidValue;
    Prob<T> P = make_prob<T>(ctx);
    const long long rows = (long long)ctx->N * ctx->G;
    const int bx = (int)std::min<long long>((ctx->Nc + 255) / 256, 32);
    const int by = (int)std::min<long long>(rows, 64);  // 32 x 64 CTAs stride over the rows
    k_chi_rest_fill<T><<<dim3((unsigned)bx, (unsigned)by), 256, 0, st>>>(P, (const T *)ctx->d_chi0L, chi,
                                                                          ctx->d_chi_dirty, force ? 1 : 0);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    return cudaMemsetAsync(ctx->d_chi_dirty, 0, sizeof(int), st);
}

template <class T>
cudaError_t launch_chi0(const shd_ctx *ctx, cudaStream_t st)
{
    Prob<T> P = make_prob<T>(ctx);
    long long n = ctx->Nc * ctx->G;
    k_chi0<T><<<blocks_for(n, 256), 256, 0, st>>>(P, (T *)ctx->d_chi0);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess || !ctx->d_chi0L) return e;
    k_chi0_layout<T><<<blocks_for(3 * n, 256), 256, 0, st>>>(P, (const T *)ctx->d_chi0, (T *)ctx->d_chi0L,
                                                            ctx->d_chi_dirty);
    note_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_source(const shd_ctx *ctx, const T *Ip, T *Sp, cudaStream_t st)
{
    if (ctx->scat_kind == SHD_SCAT_KN_THERMAL)
        return launch_source_thermal<T>(ctx, Ip, Sp, (const T *)ctx->d_mom, Sp, false, nullptr, st);
    Prob<T> P = make_prob<T>(ctx);
    size_t sm = (size_t)ctx->G * ctx->NLM * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(k_source<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_source<T><<<(unsigned)ctx->Nc, 256, sm, st>>>(P, Ip, Sp);
    note_launch();
    return cudaGetLastError();
}

template <class T, int NPT>
static cudaError_t launch_sweep_npt(const shd_ctx *ctx, T *I, const T *eta, const T *chi, cudaStream_t st,
                                    int threads)
{
    Prob<T> P = make_prob<T>(ctx);
    size_t sm = sweep_smem_bytes(ctx);
    cudaError_t e = cudaFuncSetAttribute(k_sweep<T, NPT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    k_sweep<T, NPT><<<(unsigned)(ctx->N * ctx->G), threads, sm, st>>>(P, I, eta, chi);
    note_launch();
    return cudaGetLastError();
}

// Optical depth of one short-characteristic step is at most s_max chi~_max
// with chi~ = chi_lab + kappa and chi_lab <= chi0_max D_max, D = Gamma - u.n <
// 2 Gamma (R17): true when that stays within kFp64Tau.
static bool sweep_tau_bounded(const shd_ctx *c)
{
    double smax = 0;
    for (const Ordinate &o : c->h_ord) smax = o.s > smax ? o.s : smax;
    const double chi = (c->h_alpha_max + c->h_ne_max * c->h_sigma_max) * 2.0 * c->h_gamma_max + c->kappa;
    return std::isfinite(chi) && smax * chi <= (double)kFp64Tau;
}

template <class T, int U, bool VEC>
static cudaError_t launch_sweep_pipe(const shd_ctx *ctx, T *I, const T *eta, const T *chi, cudaStream_t st,
                                     size_t sm, bool bits)
{
    Prob<T> P = make_prob<T>(ctx);
    const T *c0L = bits ? (const T *)ctx->d_chi0L : nullptr;
    const unsigned long long *mb = bits ? ctx->d_mbits : nullptr;
    if (bits) sm += sizeof(unsigned long long) * (size_t)ctx->mbits_npc;
    // FP64 weights are needed only if a step's optical depth can exceed kFp64Tau
    const bool wide = sizeof(T) == 4 && !sweep_tau_bounded(ctx);
    auto kern = bits ? (wide ? k_sweep_pipe<T, U, VEC, VEC, (sizeof(T) == 4)> : k_sweep_pipe<T, U, VEC, VEC, false>)
                     : (wide ? k_sweep_pipe<T, U, VEC, false, (sizeof(T) == 4)> : k_sweep_pipe<T, U, VEC, false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)(ctx->N * ctx->G), 1024, sm, st>>>(P, I, eta, chi, c0L, mb, ctx->mbits_npc, ctx->mbits_nwin);
    note_launch();
    return cudaGetLastError();
}

// shared memory of the FP32 two-buffer sweep: two float4 planes and the
// 2-stage ring of the three inputs
static size_t sweep_pp_smem_bytes(const shd_ctx *c)
{
    size_t ps = (((size_t)sweep_plane_max(c) + 3) & ~(size_t)3) + 4;  // k_sweep_pp's plane stride
    return sizeof(float) * ps * 14;
}

template <int U, int NT>
static cudaError_t launch_sweep_pp(const shd_ctx *ctx, float *I, const float *eta, const float *chi, cudaStream_t st,
                                   bool bits, bool wide, unsigned nblocks, int tune_stride)
{
    Prob<float> P = make_prob<float>(ctx);
    const float *c0L = bits ? (const float *)ctx->d_chi0L : nullptr;
    const unsigned long long *mb = bits ? ctx->d_mbits : nullptr;
    const size_t sm = sweep_pp_smem_bytes(ctx);
    auto kern = bits ? (wide ? k_sweep_pp<U, true, true, NT> : k_sweep_pp<U, true, false, NT>)
                     : (wide ? k_sweep_pp<U, false, true, NT> : k_sweep_pp<U, false, false, NT>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<nblocks, NT, sm, st>>>(P, I, eta, chi, c0L, mb, ctx->mbits_npc, ctx->mbits_nwin, tune_stride);
    note_launch();
    return cudaGetLastError();
}

// ---- schedules of the FP32 plane sweep ------------------------------------
// A schedule splits every plane over a cluster of C CTAs of NT threads, U
// nodes a thread (C = 1: k_sweep_pp, one CTA of NT = 1024, 512 or 256
// threads a plane).

struct SweepSched {
    int C = 0, NT = 0, U = 0, pstride = 0;
    size_t smem = 0;
};

// rows of a plane per CTA of a C-CTA cluster (the kernel's own rule)
static int sweep_rows_per_cta(int n1, int n2, int C)
{
    int R = (n1 + C - 1) / C;
    const int q4 = (n2 & 3) == 0 ? 1 : ((n2 & 1) == 0 ? 2 : 4);
    return (R + q4 - 1) / q4 * q4;
}

// Nodes per CTA of the largest class plane under a C-CTA split.
static int sweep_nloc_max(const shd_ctx *c, int C)
{
    const int dims[3] = {c->nx, c->ny, c->nz};
    bool seen[3] = {false, false, false};
    int m = 0;
    for (const Ordinate &o : c->h_ord) {
        if (seen[o.d]) continue;
        seen[o.d] = true;
        const int n1 = dims[o.e1], n2 = dims[o.e2];
        const int R = sweep_rows_per_cta(n1, n2, C);
        const int nl = (R < n1 ? R : n1) * n2;
        m = nl > m ? nl : m;
    }
    return m;
}

template <int U, int NT>
static cudaError_t launch_sweep_cl_t(const shd_ctx *ctx, const SweepSched &sc, float *I, const float *eta,
                                     const float *chi, cudaStream_t st, bool bits, bool wide, int nclusters,
                                     int tune_stride)
{
    Prob<float> P = make_prob<float>(ctx);
    const float *c0L = bits ? (const float *)ctx->d_chi0L : nullptr;
    const unsigned long long *mb = bits ? ctx->d_mbits : nullptr;
    auto kern = bits ? (wide ? k_sweep_cl<U, true, true, NT> : k_sweep_cl<U, true, false, NT>)
                     : (wide ? k_sweep_cl<U, false, true, NT> : k_sweep_cl<U, false, false, NT>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sc.smem);
    if (e != cudaSuccess) return e;
    // the whole unified L1 as shared memory, so that the CTAs the register
    // budget allows (three of 384 threads at 56 registers) also fit there
    e = cudaFuncSetAttribute(kern, cudaFuncAttributePreferredSharedMemoryCarveout, 100);
    if (e != cudaSuccess) return e;
    if (sc.C > 8) {  // 16-CTA clusters are beyond the portable size: opted in per kernel
        e = cudaFuncSetAttribute(kern, cudaFuncAttributeNonPortableClusterSizeAllowed, 1);
        if (e != cudaSuccess) return e;
    }
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3((unsigned)(nclusters * sc.C));
    cfg.blockDim = dim3(NT);
    cfg.dynamicSmemBytes = sc.smem;
    cfg.stream = st;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeClusterDimension;
    at[0].val.clusterDim.x = (unsigned)sc.C;
    at[0].val.clusterDim.y = 1;
    at[0].val.clusterDim.z = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    e = cudaLaunchKernelEx(&cfg, kern, P, I, eta, chi, c0L, mb, ctx->mbits_npc, ctx->mbits_nwin, sc.pstride,
                           tune_stride);
    note_launch();
    if (e != cudaSuccess) return e;
    return cudaGetLastError();
}

// Run schedule sc over `n` (ordinate, group) pairs (all of them, or every
// tune_stride-th into a scratch intensity when timing).
static cudaError_t run_sweep_sched(const shd_ctx *ctx, const SweepSched &sc, float *I, const float *eta,
                                   const float *chi, cudaStream_t st, bool bits, bool wide, int n, int tune_stride)
{
    if (sc.C == 1) {
#define SHD_PP(Uv, NTv) \
    if (sc.U == Uv && sc.NT == NTv) return launch_sweep_pp<Uv, NTv>(ctx, I, eta, chi, st, bits, wide, (unsigned)n, tune_stride);
        SHD_PP(1, 1024) SHD_PP(2, 1024) SHD_PP(4, 1024)
        SHD_PP(1, 512) SHD_PP(2, 512) SHD_PP(4, 512)
        SHD_PP(1, 256) SHD_PP(2, 256) SHD_PP(4, 256)
#undef SHD_PP
        return cudaErrorInvalidConfiguration;
    }
#define SHD_CL(NTv, Uv) \
    if (sc.NT == NTv && sc.U == Uv) return launch_sweep_cl_t<Uv, NTv>(ctx, sc, I, eta, chi, st, bits, wide, n, tune_stride);
    SHD_CL(256, 2) SHD_CL(256, 4) SHD_CL(384, 3) SHD_CL(512, 2) SHD_CL(512, 4) SHD_CL(768, 3) SHD_CL(1024, 2)
    SHD_CL(1024, 4)
#undef SHD_CL
    return cudaErrorInvalidConfiguration;
}

// The schedule (C, NT) with its U, buffer stride and shared memory, if it
// fits this problem; false otherwise.
template <class T>
static bool sweep_vec(const shd_ctx *ctx);

static bool sweep_sched_make(const shd_ctx *c, int C, int NT, SweepSched &sc)
{
    sc = SweepSched();
    const size_t limit = 227 * 1024;
    if (C == 1) {  // any grid: k_sweep_pp copies unaligned planes as their aligned cover
        if (NT != 1024 && NT != 512 && NT != 256) return false;
        const int pm = sweep_plane_max(c);
        const int u = (pm + NT - 1) / NT;
        if (u > 4 || sweep_pp_smem_bytes(c) > limit) return false;
        // smaller CTAs only where they keep more than half their threads busy
        if (NT < 1024 && pm <= NT / 2) return false;
        if (NT < 1024 && (1024 / NT) * sweep_pp_smem_bytes(c) > limit) return false;  // their CTAs share the SM
        sc.C = 1; sc.NT = NT; sc.U = u <= 1 ? 1 : (u <= 2 ? 2 : 4);
        sc.smem = sweep_pp_smem_bytes(c);
        return true;
    }
    if (C != 2 && C != 4 && C != 8 && C != 16) return false;
    if (!sweep_vec<float>(c)) return false;  // the cluster sweep's blocks need 16-byte aligned planes
    if (NT != 256 && NT != 384 && NT != 512 && NT != 768 && NT != 1024) return false;
    const int nl = sweep_nloc_max(c, C);
    int U = 0;
    if (NT == 384 || NT == 768) {
        // three nodes a thread: blocks that 2 or 4 a thread would fit loosely
        // (1152 nodes: 384 x 3 exactly, against 512 x 4 with a third idle)
        if (nl <= 2 * NT || nl > 3 * NT) return false;
        U = 3;
    } else if (nl <= 2 * NT) U = 2;
    else if (nl <= 4 * NT) U = 4;
    else return false;
    if (nl <= NT / 2) return false;  // half the threads or more would idle
    sc.C = C; sc.NT = NT; sc.U = U;
    sc.pstride = (nl + 3) & ~3;
    sc.smem = sizeof(float) * (size_t)sc.pstride * 14;
    return sc.smem <= limit;
}

// Every schedule that fits, k_sweep_pp's first.
static std::vector<SweepSched> sweep_candidates(const shd_ctx *c)
{
    std::vector<SweepSched> v;
    SweepSched sc;
    if (sweep_sched_make(c, 1, 1024, sc)) v.push_back(sc);
    for (int NT : {512, 256})
        if (sweep_sched_make(c, 1, NT, sc)) v.push_back(sc);
    for (int C : {2, 4, 8, 16})
        for (int NT : {256, 384, 512, 768, 1024})
            if (sweep_sched_make(c, C, NT, sc)) v.push_back(sc);
    return v;
}

// The FP32 sweep's schedule: forced, chosen earlier, or chosen now by timing
// each candidate (one warm-up and three timed launches over every
// tune_stride-th pair, intensity in a scratch array) when the stream is not
// being captured; under capture without a choice, the first candidate.
static bool sweep_schedule(const shd_ctx *cc, cudaStream_t st, const float *eta, const float *chi, bool bits,
                           bool wide, SweepSched &out)
{
    shd_ctx *c = const_cast<shd_ctx *>(cc);  // the choice is a cache of the context
    if (c->sweep_force_C > 0) return sweep_sched_make(c, c->sweep_force_C, c->sweep_force_NT, out);
    if (c->sweep_C > 0 && sweep_sched_make(c, c->sweep_C, c->sweep_NT, out)) return true;
    std::vector<SweepSched> cand = sweep_candidates(c);
    if (cand.empty()) return false;
    out = cand[0];
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) != cudaSuccess || cs != cudaStreamCaptureStatusNone) return true;
    c->sweep_ntune = 0;
    if (cand.size() > 1) {
        int sms = 0;
        if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms <= 0)
            sms = 148;
        const int npairs = c->N * c->G;
        const int n = npairs < 4 * sms ? npairs : 4 * sms;
        const int stride = npairs / n;
        float *scratch = nullptr;
        // (+16 bytes: the aligned cover of an unaligned last plane)
        if (cudaMalloc(&scratch, sizeof(float) * (size_t)n * c->Nc + 16) != cudaSuccess) {
            cudaGetLastError();
            return true;  // no room to time them: the first candidate
        }
        cudaMemsetAsync(scratch, 0, sizeof(float) * (size_t)n * c->Nc, st);
        cudaEvent_t e0, e1;
        cudaEventCreate(&e0);
        cudaEventCreate(&e1);
        float best = 1e30f;
        for (const SweepSched &sc : cand) {
            float ms = 1e30f;
            if (run_sweep_sched(c, sc, scratch, eta, chi, st, bits, wide, n, stride) == cudaSuccess) {
                cudaEventRecord(e0, st);
                bool ok = true;
                for (int r = 0; r < 3 && ok; ++r)
                    ok = run_sweep_sched(c, sc, scratch, eta, chi, st, bits, wide, n, stride) == cudaSuccess;
                cudaEventRecord(e1, st);
                if (ok && cudaEventSynchronize(e1) == cudaSuccess) {
                    cudaEventElapsedTime(&ms, e0, e1);
                    ms /= 3.f;
                }
            }
            cudaGetLastError();  // a candidate that cannot launch here is skipped
            if (c->sweep_ntune < 16) {
                c->sweep_tune[c->sweep_ntune][0] = (float)sc.C;
                c->sweep_tune[c->sweep_ntune][1] = (float)sc.NT;
                c->sweep_tune[c->sweep_ntune][2] = ms;
                c->sweep_ntune++;
            }
            if (ms < best) {
                best = ms;
                out = sc;
            }
        }
        cudaEventDestroy(e0);
        cudaEventDestroy(e1);
        cudaFree(scratch);
    }
    c->sweep_C = out.C;
    c->sweep_NT = out.NT;
    return true;
}

// shared memory of the pipelined sweep: previous plane (4 reals a node in
// FP32, 3 in FP64) + 2-stage ring of the three inputs, each array padded to
// a multiple of 4 reals
size_t sweep_pipe_smem_bytes(const shd_ctx *c)
{
    size_t ps = ((size_t)sweep_plane_max(c) + 3) & ~(size_t)3;
    return c->esize * ps * (c->esize == 4 ? 10 : 9);
}

// 16-byte copies when every plane and the array base stay 16-byte aligned
template <class T>
static bool sweep_vec(const shd_ctx *ctx)
{
    constexpr int V = 16 / sizeof(T);
    return ctx->Nc % V == 0 && ((long long)ctx->nx * ctx->ny) % V == 0 && ((long long)ctx->ny * ctx->nz) % V == 0 &&
           ((long long)ctx->nx * ctx->nz) % V == 0;
}

size_t sweep_batch_smem(const shd_ctx *c) { return sweep_pp_smem_bytes(c); }

// the descriptor of problem c as its own sweep launch would see it
void sweep_batch_fill(const shd_ctx *c, SweepBatchProb &d, long long item0)
{
    d.P = make_prob<float>(c);
    d.I = (float *)c->d_I;
    d.eta = (const float *)c->d_eta;
    d.chi = (const float *)c->d_chi;
    const bool bits = sweep_uses_chi0L<float>(c);
    d.chi0L = bits ? (const float *)c->d_chi0L : nullptr;
    d.mbits = bits ? c->d_mbits : nullptr;
    d.npc = c->mbits_npc;
    d.nwin = c->mbits_nwin;
    d.cb = bits ? 1 : 0;
    d.wide = sweep_tau_bounded(c) ? 0 : 1;
    d.item0 = item0;
}

int sweep_batch_class(const shd_ctx *c)
{
    if (c->precision == SHD_FP64 || c->integrator != SHD_SC_LINEAR) return 0;
    SweepSched sc;
    if (!sweep_sched_make(c, 1, 1024, sc)) return 0;
    if (c->sweep_force_C > 0 && !(c->sweep_force_C == 1 && c->sweep_force_NT == 1024)) return 0;
    if (c->sweep_force_C <= 0 && c->sweep_C > 0 && !(c->sweep_C == 1 && c->sweep_NT == 1024)) {
        // another schedule won the problem's timing: it joins only if the
        // 1024-thread one-CTA sweep (the batch's) timed within 3 % of that
        float pp = -1.f, best = 1e30f;
        for (int k = 0; k < c->sweep_ntune; ++k) {
            if (c->sweep_tune[k][0] == 1.f && c->sweep_tune[k][1] == 1024.f) pp = c->sweep_tune[k][2];
            best = fminf(best, c->sweep_tune[k][2]);
        }
        if (!(pp > 0.f && pp <= 1.03f * best)) return 0;
    }
    // class: U (bits 0-2), chi0 table (bit 3), FP64 weights (bit 4)
    return sc.U | (sweep_uses_chi0L<float>(c) ? 8 : 0) | (sweep_tau_bounded(c) ? 0 : 16);
}

cudaError_t launch_sweep_batch(int cls, const SweepBatchProb *d_probs, int nprob, long long nitems, size_t smem,
                               int device, cudaStream_t st)
{
    if (nprob <= 0 || nitems <= 0) return cudaSuccess;
    using KB = void (*)(const SweepBatchProb *, int, long long);
    const int U = cls & 7;
    const bool cb = (cls & 8) != 0, wide = (cls & 16) != 0;
    KB kern;
    if (U <= 1) kern = cb ? (wide ? k_sweep_batch<1, true, true> : k_sweep_batch<1, true, false>)
                          : (wide ? k_sweep_batch<1, false, true> : k_sweep_batch<1, false, false>);
    else if (U <= 2) kern = cb ? (wide ? k_sweep_batch<2, true, true> : k_sweep_batch<2, true, false>)
                               : (wide ? k_sweep_batch<2, false, true> : k_sweep_batch<2, false, false>);
    else kern = cb ? (wide ? k_sweep_batch<4, true, true> : k_sweep_batch<4, true, false>)
                   : (wide ? k_sweep_batch<4, false, true> : k_sweep_batch<4, false, false>);
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int nsm = 0, per = 0;
    if (cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, device) != cudaSuccess || nsm <= 0) nsm = 148;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, kern, 1024, smem) != cudaSuccess || per < 1) per = 1;
    long long grid = (long long)nsm * per;  // persistent: every CTA that fits at once
    if (grid > nitems) grid = nitems;
    kern<<<(unsigned)grid, 1024, smem, st>>>(d_probs, nprob, nitems);
    note_launch();
    return cudaGetLastError();
}

// (C, NT) is a schedule of the FP32 plane sweep for this problem
bool sweep_schedule_valid(const shd_ctx *c, int C, int NT)
{
    SweepSched sc;
    return c->precision != SHD_FP64 && sweep_sched_make(c, C, NT, sc);
}

template <class T>
bool sweep_uses_chi0L(const shd_ctx *ctx)
{
    if (ctx->integrator != SHD_SC_LINEAR) return false;  // the Bezier sweep reads every chi_lab
    const int u = (sweep_plane_max(ctx) + 1023) / 1024;
    return ctx->d_chi0L && ctx->d_mbits && sweep_vec<T>(ctx) && u <= 8 &&
           sweep_pipe_smem_bytes(ctx) + sizeof(unsigned long long) * (size_t)ctx->mbits_npc <= 227 * 1024;
}

// use_chi0L: the per-ordinate chi is only valid on the pieces that hold a
// moving node (the stepping path); otherwise every chi value is read.
// shared memory of the Bezier sweep: (I, S~, chi~, dS/dtau) of the previous
// plane and (S~, chi~) of the next, two slots each
size_t sweep_bez_smem_bytes(const shd_ctx *c)
{
    const size_t ps = ((size_t)sweep_plane_max(c) + 3) & ~(size_t)3;
    return c->esize * ps * 12;
}

template <class T, int U>
static cudaError_t launch_sweep_bez_u(const shd_ctx *ctx, T *I, const T *eta, const T *chi, cudaStream_t st)
{
    Prob<T> P = make_prob<T>(ctx);
    const size_t sm = sweep_bez_smem_bytes(ctx);
    const int pstride = (int)(((size_t)sweep_plane_max(ctx) + 3) & ~(size_t)3);
    const bool wide = sizeof(T) == 4 && !sweep_tau_bounded(ctx);
    auto kern = wide ? k_sweep_bez<T, U, (sizeof(T) == 4)> : k_sweep_bez<T, U, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)(ctx->N * ctx->G), 1024, sm, st>>>(P, I, eta, chi, pstride);
    note_launch();
    return cudaGetLastError();
}

// The Bezier sweep fits: planes of at most 4096 nodes within shared memory.
bool sweep_bez_usable(const shd_ctx *c)
{
    return sweep_plane_max(c) <= 4096 && sweep_bez_smem_bytes(c) <= 227 * 1024;
}

template <class T>
cudaError_t launch_sweep(const shd_ctx *ctx, T *I, const T *eta, const T *chi, cudaStream_t st, bool use_chi0L)
{
    int plane = sweep_plane_max(ctx);
    if (ctx->integrator == SHD_SC_BEZIER) {
        if (!sweep_bez_usable(ctx)) return cudaErrorInvalidConfiguration;
        const int u = (plane + 1023) / 1024;
        if (u <= 1) return launch_sweep_bez_u<T, 1>(ctx, I, eta, chi, st);
        if (u <= 2) return launch_sweep_bez_u<T, 2>(ctx, I, eta, chi, st);
        return launch_sweep_bez_u<T, 4>(ctx, I, eta, chi, st);
    }
    size_t smp = sweep_pipe_smem_bytes(ctx);
    if constexpr (sizeof(T) == 4) {
        {
            const bool bits = use_chi0L && sweep_uses_chi0L<T>(ctx);
            const bool wide = !sweep_tau_bounded(ctx);
            SweepSched sc;
            if (sweep_schedule(ctx, st, (const float *)eta, (const float *)chi, bits, wide, sc))
                return run_sweep_sched(ctx, sc, (float *)I, (const float *)eta, (const float *)chi, st, bits, wide,
                                       ctx->N * ctx->G, 0);
        }
    }
    if (smp <= 227 * 1024) {
        const bool vec = sweep_vec<T>(ctx);
        const bool bits = use_chi0L && sweep_uses_chi0L<T>(ctx);
        int u = (plane + 1023) / 1024;
        if (vec) {
            if (u <= 1) return launch_sweep_pipe<T, 1, true>(ctx, I, eta, chi, st, smp, bits);
            if (u <= 2) return launch_sweep_pipe<T, 2, true>(ctx, I, eta, chi, st, smp, bits);
            if (u <= 4) return launch_sweep_pipe<T, 4, true>(ctx, I, eta, chi, st, smp, bits);
            if (u <= 8) return launch_sweep_pipe<T, 8, true>(ctx, I, eta, chi, st, smp, bits);
        } else {
            if (u <= 1) return launch_sweep_pipe<T, 1, false>(ctx, I, eta, chi, st, smp, false);
            if (u <= 2) return launch_sweep_pipe<T, 2, false>(ctx, I, eta, chi, st, smp, false);
            if (u <= 4) return launch_sweep_pipe<T, 4, false>(ctx, I, eta, chi, st, smp, false);
            if (u <= 8) return launch_sweep_pipe<T, 8, false>(ctx, I, eta, chi, st, smp, false);
        }
    }
    int threads = plane < 1024 ? ((plane + 31) / 32) * 32 : 1024;
    int npt = (plane + threads - 1) / threads;
    if (npt <= 1) return launch_sweep_npt<T, 1>(ctx, I, eta, chi, st, threads);
    if (npt <= 2) return launch_sweep_npt<T, 2>(ctx, I, eta, chi, st, threads);
    if (npt <= 4) return launch_sweep_npt<T, 4>(ctx, I, eta, chi, st, threads);
    if (npt <= 8) return launch_sweep_npt<T, 8>(ctx, I, eta, chi, st, threads);
    if (npt <= 16) return launch_sweep_npt<T, 16>(ctx, I, eta, chi, st, threads);
    return cudaErrorInvalidConfiguration;
}

template <class T>
cudaError_t launch_sums(shd_ctx *ctx, const T *mom, const T *Sp, const T *Sprev, bool have_prev, cudaStream_t st)
{
    Prob<T> P = make_prob<T>(ctx);
    int nb = ctx->n_partial;
    k_sums_partial<T><<<nb, 256, 0, st>>>(P, mom, Sp, Sprev, have_prev ? 1 : 0, ctx->d_partial);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_sums_final<<<1, kSumsThreads, 0, st>>>(ctx->d_partial, nb, have_prev ? 1 : 0, ctx->d_sums);
    note_launch();
    return cudaGetLastError();
}

static int source_thermal_warps(const shd_ctx *c, size_t *sm);

// k_source_kn: shared memory at tile size tn (the transposed K, two tiles of
// I_lm, with ps two of S_prev, the tile's factors), and the largest tile size
// (8, 4 or 2 nodes) that fits; 0 where the kernel does not apply (G NLM not
// a multiple of 4, more than 64 groups) and k_source_sums takes over.
static size_t source_kn_smem(const shd_ctx *c, int tn, bool ps)
{
    const size_t G4 = 4 * (size_t)((c->G + 3) / 4);
    return sizeof(float) * ((size_t)(c->L + 1) * c->G * G4 + (size_t)(ps ? 4 : 2) * tn * c->G * c->NLM +
                            (size_t)2 * tn * G4);
}
// the largest tile first, with S_prev in shared memory where that still fits
// (a smaller tile costs more than the prefetch saves); 0: k_source_sums
static int source_kn_tile(const shd_ctx *c, bool &ps)
{
    ps = false;
    if (((long long)c->G * c->NLM) % 4 != 0 || c->G > 64) return 0;
    for (int tn : {8, 4, 2}) {
        for (bool p : {true, false})
            if (source_kn_smem(c, tn, p) <= 227 * 1024) {
                ps = p;
                return tn;
            }
    }
    return 0;
}

// k_source_kn_th: shared memory at tile size tn (two transposed tables, two
// tiles, the tile's factors and weights), and the largest tile size (4 or 2)
// that fits; 0 where k_source_thermal takes over.
static size_t source_kn_th_smem(const shd_ctx *c, int tn)
{
    const size_t G4 = 4 * (size_t)((c->G + 3) / 4);
    return sizeof(float) * ((size_t)2 * (c->L + 1) * c->G * G4 + (size_t)2 * tn * c->G * c->NLM +
                            (size_t)2 * tn * G4 + (size_t)tn);
}
static int source_kn_th_tile(const shd_ctx *c)
{
    if (((long long)c->G * c->NLM) % 4 != 0 || c->G > 64) return 0;
    for (int tn : {4, 2})
        if (source_kn_th_smem(c, tn) <= 227 * 1024) return tn;
    return 0;
}

static size_t source_sums_smem(const shd_ctx *c)
{
    return c->esize * ((((size_t)(c->L + 1) * (c->G * c->G + 1)) + 1 & ~(size_t)1) + (size_t)8 * c->G * c->NLM);
}

template <class T>
bool source_sums_usable(const shd_ctx *ctx)
{
    if (ctx->scat_kind == SHD_SCAT_KN_THERMAL) return source_thermal_warps(ctx, nullptr) > 0;
    return source_sums_smem(ctx) <= 227 * 1024;
}

// a2 and the a5 partials in one pass (see k_source_sums), then k_sums_final.
template <class T>
cudaError_t launch_source_sums(shd_ctx *ctx, const T *Ip, T *Sp, const T *mom, const T *Sprev, bool have_prev,
                               cudaStream_t st)
{
    if (ctx->scat_kind == SHD_SCAT_KN_THERMAL) {
        int grid = 0;
        cudaError_t e = launch_source_thermal<T>(ctx, Ip, Sp, mom, Sprev, have_prev, &grid, st);
        if (e != cudaSuccess) return e;
        k_sums_final<<<1, kSumsThreads, 0, st>>>(ctx->d_partial, grid, have_prev ? 1 : 0, ctx->d_sums);
        note_launch();
        return cudaGetLastError();
    }
    Prob<T> P = make_prob<T>(ctx);
    const size_t sm = source_sums_smem(ctx);
    auto kern = ctx->k_diagonal && ctx->G <= 32 ? k_source_sums<T, true> : k_source_sums<T, false>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    const int nb = ctx->n_partial;
    int grid_cc = nb;  // partial-sum rows of the CUDA-core pass
    auto cuda_cores = [&]() -> cudaError_t {
        if constexpr (sizeof(T) == 4) {
            bool ps = false;
            const int tn = ctx->k_diagonal && ctx->G <= 32 ? 0 : source_kn_tile(ctx, ps);
            if (tn > 0) {
                const size_t smk = source_kn_smem(ctx, tn, ps);
                auto kk = tn == 8 ? (ps ? k_source_kn<8, true> : k_source_kn<8, false>)
                                  : (tn == 4 ? (ps ? k_source_kn<4, true> : k_source_kn<4, false>)
                                             : (ps ? k_source_kn<2, true> : k_source_kn<2, false>));
                cudaError_t e2 = cudaFuncSetAttribute(kk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smk);
                if (e2 != cudaSuccess) return e2;
                const long long ntile = (ctx->Nc + tn - 1) / tn;
                const int units = ((ctx->G + 3) / 4) * ctx->NLM;
                const int nt = units >= 512 ? 512 : (units + 31) / 32 * 32;
                // persistent: as many CTAs as fit on every SM at once (few
                // groups make small CTAs, several a SM)
                int g = 0, per_sm = 0;
                if (cudaDeviceGetAttribute(&g, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || g <= 0)
                    g = 148;
                if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kk, nt, smk) != cudaSuccess || per_sm < 1)
                    per_sm = 1;
                g *= per_sm;
                if (g > nb) g = nb;
                if (ntile < g) g = (int)ntile;
                kk<<<g, nt, smk, st>>>(P, (const float *)Ip, (float *)Sp, (const float *)mom, (const float *)Sprev,
                                       have_prev ? 1 : 0, ctx->d_partial);
                note_launch();
                grid_cc = g;
                return cudaGetLastError();
            }
        }
        kern<<<nb, 256, sm, st>>>(P, Ip, Sp, mom, Sprev, have_prev ? 1 : 0, ctx->d_partial);
        note_launch();
        grid_cc = nb;
        return cudaGetLastError();
    };
    bool tc = false;
    if constexpr (sizeof(T) == 4) {
        // group-mixing kernels in the mixed precision: the tensor-core pass or
        // the CUDA-core pass, whichever ran faster when first timed (outside
        // a capture; both compute the same S_lm and partial sums)
        if (source_tc_usable(ctx)) {
            shd_ctx *c = const_cast<shd_ctx *>(ctx);  // the choice is a cache of the context
            int grid_tc = 0;
            auto tc_pass = [&]() {
                return launch_source_sums_tc(c, (const float *)Ip, (float *)Sp, (const float *)mom,
                                             (const float *)Sprev, have_prev, &grid_tc, st);
            };
            cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
            if (c->source_choice == 0 && cudaStreamIsCapturing(st, &cs) == cudaSuccess &&
                cs == cudaStreamCaptureStatusNone) {
                cudaEvent_t ev[3];
                for (auto &x : ev) cudaEventCreate(&x);
                float t_tc = 1e30f, t_cc = 1e30f;
                cudaEventRecord(ev[0], st);
                bool ok = tc_pass() == cudaSuccess;
                cudaEventRecord(ev[1], st);
                ok = ok && cuda_cores() == cudaSuccess;
                cudaEventRecord(ev[2], st);
                if (ok && cudaEventSynchronize(ev[2]) == cudaSuccess) {
                    cudaEventElapsedTime(&t_tc, ev[0], ev[1]);
                    cudaEventElapsedTime(&t_cc, ev[1], ev[2]);
                }
                for (auto &x : ev) cudaEventDestroy(x);
                cudaGetLastError();
                c->source_ms[0] = t_cc;
                c->source_ms[1] = t_tc;
                c->source_choice = t_tc < t_cc ? 2 : 1;
            }
            tc = c->source_choice == 2;
        }
    }
    int nparts = nb;  // partial-sum rows the final reduction adds
    if (tc) {
        e = launch_source_sums_tc(const_cast<shd_ctx *>(ctx), (const float *)Ip, (float *)Sp, (const float *)mom,
                                  (const float *)Sprev, have_prev, &nparts, st);
    } else {
        e = cuda_cores();
        nparts = grid_cc;
    }
    if (e != cudaSuccess) return e;
    k_sums_final<<<1, kSumsThreads, 0, st>>>(ctx->d_partial, nparts, have_prev ? 1 : 0, ctx->d_sums);
    note_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_canon_to_do(const shd_ctx *ctx, const double *src, T *dst, long long c0, long long nc,
                               cudaStream_t st)
{
    Prob<T> P = make_prob<T>(ctx);
    long long n = nc * ctx->G * ctx->N;
    if (n == 0) return cudaSuccess;
    k_canon_to_do<T><<<blocks_for(n, 256), 256, 0, st>>>(P, src, dst, c0, nc);
    note_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_do_to_canon(const shd_ctx *ctx, const T *src, double *dst, long long c0, long long nc,
                               cudaStream_t st)
{
    Prob<T> P = make_prob<T>(ctx);
    long long n = nc * ctx->G * ctx->N;
    if (n == 0) return cudaSuccess;
    k_do_to_canon<T><<<blocks_for(n, 256), 256, 0, st>>>(P, src, dst, c0, nc);
    note_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_convert(const double *src, T *dst, long long n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_convert<T><<<blocks_for(n, 256), 256, 0, st>>>(src, dst, n);
    note_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_convert_back(const T *src, double *dst, long long n, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_convert_back<T><<<blocks_for(n, 256), 256, 0, st>>>(src, dst, n);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_kn_table(int G, const double *d_edges, int L, double *d_K, double *d_sigma_out,
                            const double *d_gx, const double *d_gw, int nq, cudaStream_t st)
{
    k_kn_table<<<blocks_for((long long)G * G, 64), 64, 0, st>>>(G, d_edges, L, d_K, d_sigma_out, d_gx, d_gw, nq);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_kn_thermal_tables(int G, const double *d_edges, int L, const double *d_quad, double *d_K,
                                     double *d_so, cudaStream_t st)
{
    const size_t sm = sizeof(double) * ((size_t)(L + 1) * G + 3 * TN_S + 1);
    k_kn_thermal_table<<<(unsigned)(G * kThermalN), 256, sm, st>>>(G, d_edges, L, d_quad, d_K, d_so);
    note_launch();
    return cudaGetLastError();
}

// warps per CTA of the thermal source pass: as many as shared memory allows
static int source_thermal_warps(const shd_ctx *c, size_t *sm)
{
    const size_t per = (size_t)(c->L + 1) * c->G * c->G;
    for (int w = 8; w >= 1; w >>= 1) {
        const size_t b = c->esize * (2 * per + (size_t)w * c->G * c->NLM);
        if (b <= 227 * 1024) {
            if (sm) *sm = b;
            return w;
        }
    }
    return 0;
}

template <class T>
cudaError_t launch_source_thermal(const shd_ctx *ctx, const T *Ip, T *Sp, const T *mom, const T *Sprev,
                                  bool have_prev, int *grid_used, cudaStream_t st)
{
    Prob<T> P = make_prob<T>(ctx);
    if constexpr (sizeof(T) == 4) {
        // the register-blocked form where its two tables and tiles fit
        const int tn = source_kn_th_tile(ctx);
        if (tn > 0 && P.thermal) {
            const size_t smk = source_kn_th_smem(ctx, tn);
            auto kk = tn == 4 ? k_source_kn_th<4> : k_source_kn_th<2>;
            cudaError_t e2 = cudaFuncSetAttribute(kk, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smk);
            if (e2 != cudaSuccess) return e2;
            const int units = ((ctx->G + 3) / 4) * ctx->NLM;
            const int nt = units >= 512 ? 512 : (units + 31) / 32 * 32;
            int g = 0, per_sm = 0;
            if (cudaDeviceGetAttribute(&g, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || g <= 0)
                g = 148;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, kk, nt, smk) != cudaSuccess || per_sm < 1)
                per_sm = 1;
            g *= per_sm;
            if (g > ctx->n_partial) g = ctx->n_partial;
            if (g > ctx->nthchunk) g = ctx->nthchunk;
            if (g < 1) g = 1;
            kk<<<g, nt, smk, st>>>(P, (const float *)Ip, (float *)Sp, (const float *)mom, (const float *)Sprev,
                                   have_prev ? 1 : 0, ctx->d_partial);
            note_launch();
            if (grid_used) *grid_used = g;
            return cudaGetLastError();
        }
    }
    size_t sm = 0;
    const int W = source_thermal_warps(ctx, &sm);
    if (W == 0 || !P.thermal) return cudaErrorInvalidConfiguration;
    cudaError_t e = cudaFuncSetAttribute(k_source_thermal<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    int grid = ctx->nthchunk < ctx->n_partial ? ctx->nthchunk : ctx->n_partial;
    if (grid < 1) grid = 1;
    k_source_thermal<T><<<grid, 32 * W, sm, st>>>(P, Ip, Sp, mom, Sprev, have_prev ? 1 : 0, ctx->d_partial);
    note_launch();
    if (grid_used) *grid_used = grid;
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_ng_dots(const T *x0, const T *x1, const T *x2, const T *x3, long long n, double *part, int nblk,
                           double *out5, cudaStream_t st)
{
    k_ng_dots<T><<<nblk, kNgThreads, 0, st>>>(x0, x1, x2, x3, n, part);
    note_launch();
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return e;
    k_ng_final<<<1, kNgThreads, 0, st>>>(part, nblk, out5);
    note_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_ng_combine(T *x0, const T *x1, const T *x2, long long n, double a, double b, cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_ng_combine<T><<<blocks_for(n, 256), 256, 0, st>>>(x0, x1, x2, n, a, b);
    note_launch();
    return cudaGetLastError();
}

template <class T>
cudaError_t launch_rk_stage(T *I, const T *A, T *B, T *acc, long long n, double cnext, bool first, bool last,
                            cudaStream_t st)
{
    if (n == 0) return cudaSuccess;
    k_rk_stage<T><<<blocks_for(n, 256), 256, 0, st>>>(I, A, B, acc, n, (T)cnext, first ? 1 : 0, last ? 1 : 0);
    note_launch();
    return cudaGetLastError();
}

#define SHD_INSTANTIATE(T)                                                                                  \
    template Prob<T> make_prob<T>(const shd_ctx *);                                                         \
    template cudaError_t launch_chi0<T>(const shd_ctx *, cudaStream_t);                                     \
    template cudaError_t launch_source<T>(const shd_ctx *, const T *, T *, cudaStream_t);                   \
    template cudaError_t launch_sweep<T>(const shd_ctx *, T *, const T *, const T *, cudaStream_t, bool);   \
    template cudaError_t launch_chi_rest_fill<T>(const shd_ctx *, T *, cudaStream_t, bool);                   \
    template bool sweep_uses_chi0L<T>(const shd_ctx *);                                                     \
    template cudaError_t launch_sums<T>(shd_ctx *, const T *, const T *, const T *, bool, cudaStream_t);    \
    template cudaError_t launch_source_sums<T>(shd_ctx *, const T *, T *, const T *, const T *, bool,       \
                                               cudaStream_t);                                               \
    template bool source_sums_usable<T>(const shd_ctx *);                                                   \
    template cudaError_t launch_canon_to_do<T>(const shd_ctx *, const double *, T *, long long, long long,  \
                                               cudaStream_t);                                               \
    template cudaError_t launch_do_to_canon<T>(const shd_ctx *, const T *, double *, long long, long long,  \
                                               cudaStream_t);                                               \
    template cudaError_t launch_convert<T>(const double *, T *, long long, cudaStream_t);                   \
    template cudaError_t launch_convert_back<T>(const T *, double *, long long, cudaStream_t);               \
    template cudaError_t launch_ng_dots<T>(const T *, const T *, const T *, const T *, long long, double *,  \
                                           int, double *, cudaStream_t);                                    \
    template cudaError_t launch_ng_combine<T>(T *, const T *, const T *, long long, double, double,         \
                                              cudaStream_t);                                                \
    template cudaError_t launch_rk_stage<T>(T *, const T *, T *, T *, long long, double, bool, bool,         \
                                            cudaStream_t);                                                  \
    template cudaError_t launch_source_thermal<T>(const shd_ctx *, const T *, T *, const T *, const T *,     \
                                                  bool, int *, cudaStream_t);

SHD_INSTANTIATE(double)
SHD_INSTANTIATE(float)

}  // namespace shd
