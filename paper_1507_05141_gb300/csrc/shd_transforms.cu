// Stages a1 (project) and a3 (sh2lab) as node-tiled contractions on CUDA
// cores, plus the Lorentz remaps of moving nodes (Sec. 2.2).
//
// A node tile is an 8 x 8 brick in (x, y) at one z.  In every sweep layout
// (see shd_internal.cuh) such a brick is 8 contiguous runs of 8 nodes, so the
// tile of one (ordinate, group) is read or written as eight 32-byte runs.
//
//   a1  I_lm(c,g)  = sum_k W_k Y_p(n_k) I0(c,k,g)          (Sec. 2.3 SH)
//       moments    = sum_k W_k {1, n_i, n_i n_j}/(4 pi) I(c,k,g)
//     as one contraction per (tile, g): [64 nodes x N] x [N x (NLM + 10)].
//     For a moving node I0 is the comoving intensity from k_remap_to_comoving
//     (in the scratch buffer); its moments still use the laboratory I.
//   a3  S0(c,k,g)  = sum_p Y_p(n_k) S_p(c,g)   per (tile, g): [64 x NLM] x [NLM x N];
//     a node at rest writes eta = chi0 S0, chi = chi0 directly; a moving node
//     writes S0 to the scratch buffer and k_remap_to_lab does the transform.
//
// The remaps (one CTA per moving node, its G x N values in shared memory)
// are shared by every precision.  In single precision they read each
// (node, ordinate)'s boosted stencil and Doppler ratio from the tables that
// k_remap_tables builds once per flow field, and with group centres equally
// spaced in log energy they replace the bracket search by a constant shift.
#include <cuda_runtime.h>

#include <type_traits>

#include "shd_internal.cuh"

namespace shd {

__device__ inline int tile_row(int d, int q)
{
    // element q of a run-ordered brick -> row r = (iy - y0)*8 + (ix - x0);
    // runs follow x for the z- and y-dominant layouts and y for the x-dominant one
    return d == 0 ? ((q & 7) << 3) | (q >> 3) : q;
}

// -------------------------------------------------------------------------
// a1: [64 x N] x [N x NB] per (tile, group); 128 threads = 8 row groups of 8
// rows x 16 column groups of TC columns (NB = 16 TC >= NLM + 10).
// -------------------------------------------------------------------------
template <class T, int TC>
__global__ void __launch_bounds__(128) k_project_tile(Prob<T> P, const T *__restrict__ I, const T *__restrict__ I0,
                                                      T *__restrict__ Ip, T *__restrict__ mom)
{
    constexpr int R = 64, KC = 32, NB = 16 * TC, TR = 8;
    __shared__ T As[KC][R];
    __shared__ T Bs[KC][NB];
    const int tile = blockIdx.x / P.G, g = blockIdx.x - (blockIdx.x / P.G) * P.G;
    const TileInfo ti = P.tiles[tile];
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    const int NLM = P.NLM;
    const int passes = (ti.flags & 1) ? 2 : 1;
    for (int pass = 0; pass < passes; ++pass) {
        T acc[TR][TC];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TC; ++j) acc[i][j] = T(0);
        for (int k0 = 0; k0 < P.N; k0 += KC) {
            for (int e = tid; e < KC * R; e += 128) {
                int kk = e >> 6, q = e & 63, k = k0 + kk;
                T v = T(0);
                int r = q;
                if (k < P.N) {
                    int d = P.ord[k].d;
                    r = tile_row(d, q);
                    int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
                    if (ix < P.nx && iy < P.ny) {
                        const int m = P.midx[((long long)ti.z * P.ny + iy) * P.nx + ix];
                        if (pass == 1 && m >= 0)
                            v = I0[((long long)m * P.G + g) * P.N + k];  // comoving, node-major
                        else
                            v = I[((long long)k * P.G + g) * P.Nc + perm_offset(d, ix, iy, ti.z, P.nx, P.ny, P.nz)];
                    }
                }
                As[kk][r] = v;
            }
            for (int e = tid; e < KC * NB; e += 128) {
                int kk = e / NB, j = e - kk * NB, k = k0 + kk;
                Bs[kk][j] = k < P.N ? P.Bproj[(size_t)k * NB + j] : T(0);
            }
            __syncthreads();
#pragma unroll 4
            for (int kk = 0; kk < KC; ++kk) {
                T a[TR], b[TC];
#pragma unroll
                for (int i = 0; i < TR; ++i) a[i] = As[kk][tr * TR + i];
#pragma unroll
                for (int j = 0; j < TC; ++j) b[j] = Bs[kk][tc + 16 * j];
#pragma unroll
                for (int i = 0; i < TR; ++i)
#pragma unroll
                    for (int j = 0; j < TC; ++j) acc[i][j] += a[i] * b[j];
            }
            __syncthreads();
        }
#pragma unroll
        for (int i = 0; i < TR; ++i) {
            int r = tr * TR + i;
            int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
            if (ix >= P.nx || iy >= P.ny) continue;
            long long c = ((long long)ti.z * P.ny + iy) * P.nx + ix;
            bool moving = P.mflag[c] != 0;
#pragma unroll
            for (int j = 0; j < TC; ++j) {
                int col = tc + 16 * j;
                if (col < NLM) {
                    if ((pass == 0 && !moving) || (pass == 1 && moving)) Ip[(c * P.G + g) * NLM + col] = acc[i][j];
                } else if (col < NLM + 10 && pass == 0) {
                    mom[(c * P.G + g) * 10 + (col - NLM)] = acc[i][j];
                }
            }
        }
    }
}

// -------------------------------------------------------------------------
// a3: [64 x NLM] x [NLM x N] per (tile, group), N in chunks of 128
// ordinates; 256 threads = 8 row groups of 8 rows x 32 column groups of 4.
// -------------------------------------------------------------------------
template <class T>
__global__ void __launch_bounds__(256) k_sh2lab_tile(Prob<T> P, const T *__restrict__ Sp, T *__restrict__ eta,
                                                     T *__restrict__ chi, T *__restrict__ S0)
{
    constexpr int R = 64, KC = 128, TR = 8, TC = 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NLM = P.NLM;
    T *As = reinterpret_cast<T *>(smem_raw);  // [NLM][R]
    T *Bs = As + (size_t)NLM * R;             // [NLM][KC]
    T *Cs = Bs + (size_t)NLM * KC;            // [KC][R + 1]
    T *chir = Cs + (size_t)KC * (R + 1);      // [R]
    int *mrow = reinterpret_cast<int *>(chir + R);  // [R] moving index of the row, -1 at rest
    const int tile = blockIdx.x / P.G, g = blockIdx.x - (blockIdx.x / P.G) * P.G;
    const TileInfo ti = P.tiles[tile];
    const int tid = threadIdx.x, tr = tid >> 5, tc = tid & 31;

    for (int e = tid; e < R * NLM; e += 256) {
        int r = e / NLM, p = e - r * NLM;
        int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
        T v = T(0);
        if (ix < P.nx && iy < P.ny) {
            long long c = ((long long)ti.z * P.ny + iy) * P.nx + ix;
            v = Sp[(c * P.G + g) * NLM + p];
        }
        As[(size_t)p * R + r] = v;
    }
    for (int r = tid; r < R; r += 256) {
        int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
        T ch = T(0);
        int m = -1;
        if (ix < P.nx && iy < P.ny) {
            long long c = ((long long)ti.z * P.ny + iy) * P.nx + ix;
            ch = P.chi0[c * P.G + g];
            m = P.midx[c];
        }
        chir[r] = ch;
        mrow[r] = m;
    }
    for (int k0 = 0; k0 < P.N; k0 += KC) {
        for (int e = tid; e < KC * NLM; e += 256) {
            int kk = e / NLM, p = e - kk * NLM, k = k0 + kk;
            Bs[(size_t)p * KC + kk] = k < P.N ? P.Y[(size_t)k * NLM + p] : T(0);
        }
        __syncthreads();
        T acc[TR][TC];
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TC; ++j) acc[i][j] = T(0);
        for (int p = 0; p < NLM; ++p) {
            T a[TR], b[TC];
#pragma unroll
            for (int i = 0; i < TR; ++i) a[i] = As[(size_t)p * R + tr * TR + i];
#pragma unroll
            for (int j = 0; j < TC; ++j) b[j] = Bs[(size_t)p * KC + tc + 32 * j];
#pragma unroll
            for (int i = 0; i < TR; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j) acc[i][j] += a[i] * b[j];
        }
#pragma unroll
        for (int i = 0; i < TR; ++i)
#pragma unroll
            for (int j = 0; j < TC; ++j) Cs[(size_t)(tc + 32 * j) * (R + 1) + tr * TR + i] = acc[i][j];
        __syncthreads();
        for (int e = tid; e < KC * R; e += 256) {
            int kk = e >> 6, q = e & 63, k = k0 + kk;
            if (k >= P.N) continue;
            int d = P.ord[k].d;
            int r = tile_row(d, q);
            int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
            if (ix >= P.nx || iy >= P.ny) continue;
            T v = Cs[(size_t)kk * (R + 1) + r];
            const int m = mrow[r];
            if (m >= 0) {
                S0[((long long)m * P.G + g) * P.N + k] = v;  // comoving, node-major
            } else {
                long long a = ((long long)k * P.G + g) * P.Nc + perm_offset(d, ix, iy, ti.z, P.nx, P.ny, P.nz);
                T ch = chir[r];
                eta[a] = ch * v;
                chi[a] = ch;
            }
        }
        __syncthreads();
    }
}

// -------------------------------------------------------------------------
// Persistent forms (used when the right-hand matrix fits in shared memory):
// one CTA per SM loads W Y (project) or Y (sh2lab) once and then walks the
// (tile, group) work items, so the matrix crosses L2 once per SM instead of
// once per item.  A chunks are double-buffered with cp.async.
// -------------------------------------------------------------------------
__device__ inline void cp_async4(void *smem, const void *gmem)
{
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;\n" ::"r"(s), "l"(gmem));
}
__device__ inline void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::); }
template <int N>
__device__ inline void cp_async_wait() { asm volatile("cp.async.wait_group %0;\n" ::"n"(N)); }

// a1, persistent: 256 threads = 16 row groups of 4 rows x 16 column groups of
// TC contiguous columns (NB = 16 TC).  Shared: Bs[N][NB] + As[2][KC][64].
template <int TC>
__global__ void __launch_bounds__(256, 1) k_project_persist(Prob<float> P, const float *__restrict__ I,
                                                            const float *__restrict__ I0, float *__restrict__ Ip,
                                                            float *__restrict__ mom)
{
    constexpr int R = 64, KC = 32, NB = 16 * TC, TR = 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    float *Bs = reinterpret_cast<float *>(smem_raw);        // [N][NB]
    float *As = Bs + (size_t)P.N * NB;                       // [2][KC][R]
    const int tid = threadIdx.x, tr = tid >> 4, tc = tid & 15;
    const int NLM = P.NLM, N = P.N, G = P.G;
    for (int e = tid; e < N * NB; e += 256) Bs[e] = P.Bproj[e];
    const long long items = P.ntiles * G;
    const int nchunk = (N + KC - 1) / KC;
    for (long long w = blockIdx.x; w < items; w += gridDim.x) {
        const long long tile = w / G;
        const int g = (int)(w - tile * G);
        const TileInfo ti = P.tiles[tile];
        const int passes = (ti.flags & 1) ? 2 : 1;
        for (int pass = 0; pass < passes; ++pass) {
            // columns this pass needs: everything in pass 0, the SH part in pass 1
            const int ncol = pass == 0 ? NB : NLM;
            float acc[TR][TC];
#pragma unroll
            for (int i = 0; i < TR; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j) acc[i][j] = 0.f;
            auto load_chunk = [&](int ch, int buf) {
                float *A = As + (size_t)buf * KC * R;
                for (int e = tid; e < KC * R; e += 256) {
                    int kk = e >> 6, q = e & 63, k = ch * KC + kk;
                    int r = q;
                    bool ok = false;
                    const float *src = nullptr;
                    if (k < N) {
                        int d = P.ord[k].d;
                        r = tile_row(d, q);
                        int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
                        if (ix < P.nx && iy < P.ny) {
                            const int m = P.midx[((long long)ti.z * P.ny + iy) * P.nx + ix];
                            if (pass == 1 && m >= 0)
                                src = I0 + ((long long)m * G + g) * N + k;  // comoving, node-major
                            else
                                src = I + ((long long)k * G + g) * P.Nc + perm_offset(d, ix, iy, ti.z, P.nx, P.ny, P.nz);
                            ok = true;
                        }
                    }
                    if (ok) cp_async4(&A[kk * R + r], src);
                    else A[kk * R + r] = 0.f;
                }
                cp_async_commit();
            };
            __syncthreads();  // previous item's readers of As are done (and Bs is loaded)
            load_chunk(0, 0);
            for (int ch = 0; ch < nchunk; ++ch) {
                if (ch + 1 < nchunk) {
                    load_chunk(ch + 1, (ch + 1) & 1);
                    cp_async_wait<1>();
                } else {
                    cp_async_wait<0>();
                }
                __syncthreads();
                const float *A = As + (size_t)(ch & 1) * KC * R;
                const int kbase = ch * KC;
                const int kmax = N - kbase < KC ? N - kbase : KC;
                if (tc * TC < ncol) {
                    for (int kk = 0; kk < kmax; ++kk) {
                        float4 a4 = *reinterpret_cast<const float4 *>(&A[kk * R + tr * TR]);
                        const float *b = &Bs[(size_t)(kbase + kk) * NB + tc * TC];
                        float bv[TC];
#pragma unroll
                        for (int j = 0; j < TC; ++j) bv[j] = b[j];
                        float av[4] = {a4.x, a4.y, a4.z, a4.w};
#pragma unroll
                        for (int i = 0; i < TR; ++i)
#pragma unroll
                            for (int j = 0; j < TC; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
                    }
                }
                __syncthreads();  // buffer (ch & 1) may be refilled next
            }
#pragma unroll
            for (int i = 0; i < TR; ++i) {
                int r = tr * TR + i;
                int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
                if (ix >= P.nx || iy >= P.ny) continue;
                long long c = ((long long)ti.z * P.ny + iy) * P.nx + ix;
                bool moving = P.mflag[c] != 0;
#pragma unroll
                for (int j = 0; j < TC; ++j) {
                    int col = tc * TC + j;
                    if (col < NLM) {
                        if ((pass == 0 && !moving) || (pass == 1 && moving)) Ip[(c * G + g) * NLM + col] = acc[i][j];
                    } else if (col < NLM + 10 && pass == 0) {
                        mom[(c * G + g) * 10 + (col - NLM)] = acc[i][j];
                    }
                }
            }
        }
    }
}

// a3, persistent: Bs = Y^T [NLM][N] resident; per item As [NLM][64], the
// result staged per 128-ordinate chunk in Cs [128][65] and written as runs.
__global__ void __launch_bounds__(256, 1) k_sh2lab_persist(Prob<float> P, const float *__restrict__ Sp,
                                                           float *__restrict__ eta, float *__restrict__ chi,
                                                           float *__restrict__ S0)
{
    constexpr int R = 64, KC = 128, TR = 8, TC = 4;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int NLM = P.NLM, N = P.N, G = P.G;
    float *Bs = reinterpret_cast<float *>(smem_raw);  // [NLM][N]
    float *As = Bs + (size_t)NLM * N;                  // [NLM][R]
    float *Cs = As + (size_t)NLM * R;                  // [KC][R + 1]
    float *chir = Cs + (size_t)KC * (R + 1);           // [R]
    int *mrow = reinterpret_cast<int *>(chir + R);     // [R] moving index, -1 at rest
    const int tid = threadIdx.x, tr = tid >> 5, tc = tid & 31;
    for (int e = tid; e < N * NLM; e += 256) {
        int k = e / NLM, p = e - k * NLM;
        Bs[(size_t)p * N + k] = P.Y[e];
    }
    const long long items = P.ntiles * G;
    for (long long w = blockIdx.x; w < items; w += gridDim.x) {
        const long long tile = w / G;
        const int g = (int)(w - tile * G);
        const TileInfo ti = P.tiles[tile];
        __syncthreads();
        for (int e = tid; e < R * NLM; e += 256) {
            int r = e / NLM, p = e - r * NLM;
            int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
            float v = 0.f;
            if (ix < P.nx && iy < P.ny) {
                long long c = ((long long)ti.z * P.ny + iy) * P.nx + ix;
                v = Sp[(c * G + g) * NLM + p];
            }
            As[(size_t)p * R + r] = v;
        }
        for (int r = tid; r < R; r += 256) {
            int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
            float ch = 0.f;
            int m = -1;
            if (ix < P.nx && iy < P.ny) {
                long long c = ((long long)ti.z * P.ny + iy) * P.nx + ix;
                ch = P.chi0[c * G + g];
                m = P.midx[c];
            }
            chir[r] = ch;
            mrow[r] = m;
        }
        __syncthreads();
        for (int k0 = 0; k0 < N; k0 += KC) {
            float acc[TR][TC];
#pragma unroll
            for (int i = 0; i < TR; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j) acc[i][j] = 0.f;
            for (int p = 0; p < NLM; ++p) {
                const float *a = &As[(size_t)p * R + tr * TR];
                float4 a0 = *reinterpret_cast<const float4 *>(a);
                float4 a1 = *reinterpret_cast<const float4 *>(a + 4);
                float av[8] = {a0.x, a0.y, a0.z, a0.w, a1.x, a1.y, a1.z, a1.w};
                float bv[TC];
#pragma unroll
                for (int j = 0; j < TC; ++j) {
                    int k = k0 + tc + 32 * j;
                    bv[j] = k < N ? Bs[(size_t)p * N + k] : 0.f;
                }
#pragma unroll
                for (int i = 0; i < TR; ++i)
#pragma unroll
                    for (int j = 0; j < TC; ++j) acc[i][j] = fmaf(av[i], bv[j], acc[i][j]);
            }
#pragma unroll
            for (int i = 0; i < TR; ++i)
#pragma unroll
                for (int j = 0; j < TC; ++j) Cs[(size_t)(tc + 32 * j) * (R + 1) + tr * TR + i] = acc[i][j];
            __syncthreads();
            for (int e = tid; e < KC * R; e += 256) {
                int kk = e >> 6, q = e & 63, k = k0 + kk;
                if (k >= N) continue;
                int d = P.ord[k].d;
                int r = tile_row(d, q);
                int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
                if (ix >= P.nx || iy >= P.ny) continue;
                float v = Cs[(size_t)kk * (R + 1) + r];
                const int m = mrow[r];
                if (m >= 0) {
                    S0[((long long)m * G + g) * N + k] = v;  // comoving, node-major
                } else {
                    long long a = ((long long)k * G + g) * P.Nc + perm_offset(d, ix, iy, ti.z, P.nx, P.ny, P.nz);
                    float ch = chir[r];
                    eta[a] = ch * v;
                    chi[a] = ch;
                }
            }
            __syncthreads();
        }
    }
}

// -------------------------------------------------------------------------
// Moving nodes.  Their per-node Lorentz remaps need all (ordinate, group)
// values of one node at once, so they work on a node-major scratch
// [m][g][k] (m = index in the moving list).  Brick transposes move data
// between the sweep layout and that scratch through shared memory, both
// sides coalesced: a brick is read / written as 32-byte runs per (k, g) and
// the scratch as contiguous runs of ordinates per (m, g).
// -------------------------------------------------------------------------

// sweep layout -> node-major scratch for the moving nodes of the bricks in
// the moving-tile list; one CTA per (brick, group)
template <class T>
__global__ void __launch_bounds__(256) k_brick_to_nodes(Prob<T> P, const T *__restrict__ src, T *__restrict__ dst)
{
    constexpr int R = 64, KC = 32;
    __shared__ T S[KC][R + 1];
    __shared__ int mrow[R];
    const int tile = P.mtiles[blockIdx.x / P.G];
    const int g = blockIdx.x - (blockIdx.x / P.G) * P.G;
    const TileInfo ti = P.tiles[tile];
    const int tid = threadIdx.x;
    for (int r = tid; r < R; r += 256) {
        int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
        mrow[r] = (ix < P.nx && iy < P.ny) ? P.midx[((long long)ti.z * P.ny + iy) * P.nx + ix] : -1;
    }
    __syncthreads();
    for (int k0 = 0; k0 < P.N; k0 += KC) {
        for (int e = tid; e < KC * R; e += 256) {
            int kk = e >> 6, q = e & 63, k = k0 + kk;
            if (k >= P.N) continue;
            int d = P.ord[k].d;
            int r = tile_row(d, q);
            if (mrow[r] < 0) continue;
            int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
            S[kk][r] = src[((long long)k * P.G + g) * P.Nc + perm_offset(d, ix, iy, ti.z, P.nx, P.ny, P.nz)];
        }
        __syncthreads();
        for (int e = tid; e < R * KC; e += 256) {
            int r = e / KC, kk = e - r * KC, k = k0 + kk;
            int m = mrow[r];
            if (m >= 0 && k < P.N) dst[((long long)m * P.G + g) * P.N + k] = S[kk][r];
        }
        __syncthreads();
    }
}

// node-major scratch (two arrays) -> sweep layout, moving nodes only
template <class T>
__global__ void __launch_bounds__(256) k_nodes_to_brick(Prob<T> P, const T *__restrict__ srcA,
                                                        const T *__restrict__ srcB, T *__restrict__ dstA,
                                                        T *__restrict__ dstB)
{
    constexpr int R = 64, KC = 32;
    __shared__ T SA[KC][R + 1];
    __shared__ T SB[KC][R + 1];
    __shared__ int mrow[R];
    const int tile = P.mtiles[blockIdx.x / P.G];
    const int g = blockIdx.x - (blockIdx.x / P.G) * P.G;
    const TileInfo ti = P.tiles[tile];
    const int tid = threadIdx.x;
    for (int r = tid; r < R; r += 256) {
        int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
        mrow[r] = (ix < P.nx && iy < P.ny) ? P.midx[((long long)ti.z * P.ny + iy) * P.nx + ix] : -1;
    }
    __syncthreads();
    for (int k0 = 0; k0 < P.N; k0 += KC) {
        for (int e = tid; e < R * KC; e += 256) {
            int r = e / KC, kk = e - r * KC, k = k0 + kk;
            int m = mrow[r];
            if (m >= 0 && k < P.N) {
                long long o = ((long long)m * P.G + g) * P.N + k;
                SA[kk][r] = srcA[o];
                SB[kk][r] = srcB[o];
            }
        }
        __syncthreads();
        for (int e = tid; e < KC * R; e += 256) {
            int kk = e >> 6, q = e & 63, k = k0 + kk;
            if (k >= P.N) continue;
            int d = P.ord[k].d;
            int r = tile_row(d, q);
            if (mrow[r] < 0) continue;
            int ix = ti.x0 + (r & 7), iy = ti.y0 + (r >> 3);
            long long a = ((long long)k * P.G + g) * P.Nc + perm_offset(d, ix, iy, ti.z, P.nx, P.ny, P.nz);
            dstA[a] = SA[kk][r];
            dstB[a] = SB[kk][r];
        }
        __syncthreads();
    }
}

// Shared tables of the remap kernels: mu[nmu], lc[G], linv[G] (working
// precision) and mesh2int[N], staged once per CTA after the node's values.
template <class T>
struct RemapTables {
    T *mu, *lc, *linv;
    int *m2i;
};

template <class T>
__device__ inline RemapTables<T> remap_tables(const Prob<T> &P, unsigned char *base)
{
    RemapTables<T> t;
    t.mu = reinterpret_cast<T *>(base);
    t.lc = t.mu + P.nmu;
    t.linv = t.lc + P.G;
    t.m2i = reinterpret_cast<int *>(t.linv + P.G);
    for (int i = threadIdx.x; i < P.nmu; i += blockDim.x) t.mu[i] = P.mu[i];
    for (int i = threadIdx.x; i < P.G; i += blockDim.x) {
        t.lc[i] = P.lc[i];
        t.linv[i] = P.linv[i];
    }
    for (int i = threadIdx.x; i < P.N; i += blockDim.x) t.m2i[i] = P.mesh2int[i];
    return t;
}

// The node's G x N values (node-major, internal ordinate order) into shared
// memory, vectorised when the rows allow it.
template <class T>
__device__ inline void stage_node(T *dst, const T *src, int n)
{
    constexpr int V = 16 / sizeof(T);
    if ((reinterpret_cast<uintptr_t>(src) & 15) == 0 && (reinterpret_cast<uintptr_t>(dst) & 15) == 0 && n % V == 0) {
        // every 16-byte piece of the node in flight at once: one memory round
        // trip per CTA (the caller's barrier publishes the copies)
        const uint32_t d = (uint32_t)__cvta_generic_to_shared(dst);
        for (int i = threadIdx.x; i < n / V; i += blockDim.x)
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d + 16u * (uint32_t)i),
                         "l"(src + (size_t)i * V)
                         : "memory");
        asm volatile("cp.async.wait_all;\n" ::: "memory");
    } else {
        // B loads in flight per thread before their stores
        constexpr int B = sizeof(T) == 4 ? 8 : 4;
        const int nt = blockDim.x;
        int i = threadIdx.x;
        for (; i + (B - 1) * nt < n; i += B * nt) {
            T v[B];
#pragma unroll
            for (int j = 0; j < B; ++j) v[j] = src[i + j * nt];
#pragma unroll
            for (int j = 0; j < B; ++j) dst[i + j * nt] = v[j];
        }
        for (; i < n; i += nt) dst[i] = src[i];
    }
}

// Ring averages at the two poles (mesh rings 0 and nmu - 1, summed in mesh
// order) for every group.
// One warp per (group, ring) pair: the lanes take the ring's ordinates in
// strides of 32 and a butterfly adds their partial sums.
template <class T>
__device__ inline void pole_averages(const Prob<T> &P, const T *sv, const int *m2i, T *spole)
{
    const int lane = threadIdx.x & 31, nw = blockDim.x >> 5;
    for (int i = threadIdx.x >> 5; i < 2 * P.G; i += nw) {
        const int g = i >> 1, rr = i & 1;
        const T *F = sv + (size_t)g * P.N;
        const int base = rr ? (P.nmu - 1) * P.nphi : 0;
        T s = 0;
        for (int j = lane; j < P.nphi; j += 32) s += F[m2i[base + j]];
#pragma unroll
        for (int o = 16; o > 0; o >>= 1) s += __shfl_xor_sync(0xffffffffu, s, o);
        if (lane == 0) spole[i] = s / T(P.nphi);
    }
}

// Bilinear stencil of direction n over the (mu, phi) mesh (from the shared mu
// table), with its four ordinates given as internal indices.
template <class T>
__device__ inline Stencil<T> stencil_internal(const Prob<T> &P, const RemapTables<T> &t, const T n[3])
{
    Stencil<T> s = make_stencil<T>(t.mu, P.nmu, P.nphi, n);
#pragma unroll
    for (int i = 0; i < 4; ++i) s.k[i] = t.m2i[s.k[i]];
    return s;
}

// Stencil values of one direction per group, with the last two evaluations
// kept: consecutive output groups usually bracket neighbouring input groups.
template <class T>
struct GroupCache {
    int g0 = -1, g1 = -1;
    T v0 = 0, v1 = 0;
    __device__ inline T get(const Stencil<T> &st, const T *sv, const T *spole, int N, int g)
    {
        if (g == g1) return v1;
        if (g == g0) return v0;
        const T v = eval_stencil<T>(st, sv + (size_t)g * N, spole + 2 * g);
        g0 = g1; v0 = v1;
        g1 = g; v1 = v;
        return v;
    }
};

// Remap table entries: the stencil placement packed as mode | a << 2 | b << 12
// in the first word (a < 1024 rings, b < 2^20 phi bins), then t, tp and the
// Doppler ratio.
__device__ inline float4 table_entry(const StencilParams<float> &p, float ratio)
{
    return make_float4(__int_as_float(p.mode | (p.a << 2) | (p.b << 12)), p.t, p.tp, ratio);
}

template <class T>
__device__ inline Stencil<T> table_stencil(const float4 &e, int nphi, const int *m2i)
{
    const int code = __float_as_int(e.x);
    StencilParams<T> p;
    p.mode = code & 3;
    p.a = (code >> 2) & 1023;
    p.b = code >> 12;
    p.t = (T)e.y;
    p.tp = (T)e.z;
    Stencil<T> s = stencil_from_params<T>(p, nphi);
#pragma unroll
    for (int i = 0; i < 4; ++i) s.k[i] = m2i[s.k[i]];
    return s;
}

// One thread per (moving node m, internal ordinate k): the Lorentz boosts of
// n_k (Sec. 2.2) and the stencils of the boosted directions, as the remap
// kernels would compute them: tc for the comoving remap (n_k taken to the
// laboratory, nu/nu0), tl for the laboratory remap (n_k taken to the
// comoving frame, nu0/nu).  They depend only on the flow and the angles.
// rc, rl: the output groups whose looked-up energy (centre x the ratio) lies
// within the outer group edges, [lo, hi) packed as lo | hi << 8, decided in
// FP64 from the FP64 flow and directions.  Beyond the edges the remapped
// intensity is zero (Sec. 2.2), a jump that a single-precision ratio would
// place a rounding away from where the FP64 definition puts it.
// Within this distance of an outer edge (in group spacings, or in log
// energy for unequal groups) a single-precision lookup defers to the table's
// FP64 range: its own rounding stays below 1e-6 there.
constexpr float kEdgeTol = 1e-5f;

__device__ inline unsigned short group_range(const Prob<float> &P, double r)
{
    const int G = P.G;
    int lo = 0, hi = G;
    while (lo < G && P.centre[lo] * r < P.edges[0]) ++lo;
    while (hi > lo && P.centre[hi - 1] * r > P.edges[G]) --hi;
    return (unsigned short)(lo | (hi << 8));
}

__global__ void __launch_bounds__(256) k_remap_tables(Prob<float> P, float4 *__restrict__ tc, float4 *__restrict__ tl,
                                                      unsigned short *__restrict__ rc, unsigned short *__restrict__ rl,
                                                      const double *__restrict__ u64, const double *__restrict__ dirs64)
{
    const long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (i >= P.nmoving * P.N) return;
    const long long m = i / P.N;
    const int k = (int)(i - m * P.N);
    const long long c = P.moving[m];
    const float u[3] = {P.u[3 * c], P.u[3 * c + 1], P.u[3 * c + 2]};
    const float nk[3] = {P.dirs[3 * k], P.dirs[3 * k + 1], P.dirs[3 * k + 2]};
    float nb[3];
    const float q = boost_any<float>(u, nk, nb, -1.f, P.fp64_boost);
    tc[i] = table_entry(stencil_params<float>(P.mu, P.nmu, P.nphi, nb), q);
    const float D = boost_any<float>(u, nk, nb, 1.f, P.fp64_boost);
    tl[i] = table_entry(stencil_params<float>(P.mu, P.nmu, P.nphi, nb), D);
    const double ud[3] = {u64[3 * c], u64[3 * c + 1], u64[3 * c + 2]};
    const double nd[3] = {dirs64[3 * k], dirs64[3 * k + 1], dirs64[3 * k + 2]};
    double od[3];
    rc[i] = group_range(P, boost_dir<double>(ud, nd, od, -1.0));
    rl[i] = group_range(P, boost_dir<double>(ud, nd, od, 1.0));
}

// Energy offset x = l / (log spacing) of equally spaced log centres, split
// into its whole part s and fraction t.
template <class T>
struct UniformShift {
    T x, t;
    int s;
};

template <class T>
__device__ inline UniformShift<T> uniform_shift(const Prob<T> &P, T l)
{
    UniformShift<T> u;
    u.x = l * P.lgidl;
    const T f = dfloor<T>(u.x);
    const T lim = T(P.G + 1);  // shifts beyond the group range act alike
    u.s = (int)dclamp<T>(f, -lim, lim);
    u.t = u.x - f;
    return u;
}

// A stencil flattened for the group loop: shared-memory offsets and weights
// of the four ordinates plus the pole term, whose weight is 0 when the
// direction lies between the outer rings (the pole slot read is then finite).
template <class T>
struct FlatStencil {
    int o0, o1, o2, o3, po;
    T w0, w1, w2, w3, wp;
    // V(g) from the group-major values sv[g][N] and pole averages spole[g][2]
    __device__ inline T eval(const T *sv, const T *spole, int N, int g) const
    {
        const T *F = sv + g * N;
        T v = w0 * F[o0] + w1 * F[o1] + w2 * F[o2] + w3 * F[o3];
        return v + wp * spole[2 * g + po];
    }
};

template <class T>
__device__ inline FlatStencil<T> flat_stencil(const Stencil<T> &s)
{
    FlatStencil<T> f;
    f.o0 = s.k[0]; f.o1 = s.k[1]; f.o2 = s.k[2]; f.o3 = s.k[3];
    f.w0 = s.w[0]; f.w1 = s.w[1]; f.w2 = s.w[2]; f.w3 = s.w[3];
    f.po = s.pole_ring > 0 ? 1 : 0;
    f.wp = s.pole_ring >= 0 ? s.wpole : T(0);
    return f;
}

// lower group of an inner bracket, kept in [0, G-2]
__device__ inline int clamp_group(int ga, int G) { return ga < 0 ? 0 : (ga > G - 2 ? G - 2 : ga); }

// chi0 between centres ga and ga+1: geometric from the node's log-ratio
// table where both are positive, linear otherwise
template <class T>
__device__ inline T chi_mix(const T *schi, const T *slr, int ga, T t)
{
    const T a = schi[ga], b = schi[ga + 1];
    if (a > T(0) && b > T(0)) return freq_mix_lr<T>(a, slr[ga], t);
    return (T(1) - t) * a + t * b;
}

// laboratory I (node-major) -> comoving I0 (node-major), one CTA per moving
// node: I0(k0, g0) = (ebar_g0/eps)^3 I_lab(n, eps), n = boost of n_k0 to the
// laboratory, eps = ebar_g0 (Gamma + u.n_k0)   (Sec. 2.2)
// TAB: the boosts and stencils come from the per-flow table (FP32 only);
// otherwise they are computed in place.  Two instantiations, so that the
// table path carries none of the computed path's FP64 boost code, which the
// compiler would otherwise evaluate alongside it.
template <class T, int TAB>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 3 : 4) k_remap_to_comoving(Prob<T> P, const T *__restrict__ In, T *__restrict__ I0,
                                                           const float4 *__restrict__ tab,
                                                           const unsigned short *__restrict__ rng)
{
    static_assert(!TAB || sizeof(T) == 4, "the remap tables are FP32");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = P.G, N = P.N;
    T *sI = reinterpret_cast<T *>(smem_raw);  // [G][N] internal order
    T *spole = sI + (size_t)G * N;            // [G][2]
    const long long m = blockIdx.x;
    const long long c = P.moving[m];
    // the first two table entries of this thread, in flight during the staging
    float4 epre[2] = {};
    if constexpr (TAB) {
#pragma unroll
        for (int i = 0; i < 2; ++i) {
            const int kk = threadIdx.x + i * blockDim.x;
            if (kk < N) epre[i] = tab[m * N + kk];
        }
    }
    stage_node<T>(sI, In + m * G * N, G * N);
    const RemapTables<T> tb = remap_tables<T>(P, reinterpret_cast<unsigned char *>(spole + 2 * G));
    __syncthreads();
    pole_averages<T>(P, sI, tb.m2i, spole);
    __syncthreads();
    const T u[3] = {P.u[3 * c], P.u[3 * c + 1], P.u[3 * c + 2]};
    T *dst = I0 + m * G * N;
    int iter = 0;
    for (int k0 = threadIdx.x; k0 < N; k0 += blockDim.x, ++iter) {
        T q;  // nu/nu0
        Stencil<T> st;
        // output groups [glo, ghi) look up energies within the outer edges
        // (the table's FP64 decision; in place, the working precision's)
        // (read only for a lookup within kEdgeTol of an edge, where the
        // single-precision test could differ from the FP64 one)
        int glo = -1, ghi = -1;
        auto range = [&]() {
            if (glo < 0) {
                const unsigned r = rng[m * N + k0];
                glo = (int)(r & 255u);
                ghi = (int)(r >> 8);
            }
        };
        if constexpr (TAB) {
            const float4 e = iter == 0 ? epre[0] : (iter == 1 ? epre[1] : tab[m * N + k0]);
            q = (T)e.w;
            st = table_stencil<T>(e, P.nphi, tb.m2i);
        } else {
            T n0[3] = {P.dirs[3 * k0], P.dirs[3 * k0 + 1], P.dirs[3 * k0 + 2]};
            T n[3];
            q = boost_any<T>(u, n0, n, T(-1), P.fp64_boost);
            st = stencil_internal<T>(P, tb, n);
        }
        T iq3 = T(1) / (q * q * q);
        T lq = dlog<T>(q);
        GroupCache<T> cache;
        if (sizeof(T) == 4 && P.lgu) {
            // equally spaced log centres: energy lc[g0] + lq sits at g0 + x
            // group spacings from lc[0], x = s + t with s whole, so output
            // group g0 lies between input groups g0 + s and g0 + s + 1 at the
            // same fraction t for every g0.  Output groups below [gm0, gm1)
            // fall at or below the first centre, those above it at or beyond
            // the last.
            const FlatStencil<T> fs = flat_stencil<T>(st);
            const UniformShift<T> us = uniform_shift<T>(P, lq);
            const int gm0 = min(max(-us.s, 0), G), gm1 = max(min(G - 1 - us.s, G), gm0);
            T *out = dst + k0;
            if (gm0 > 0) {
                const T v0 = fs.eval(sI, spole, N, 0);
                for (int g0 = 0; g0 < gm0; ++g0, out += N) {
                    const T dx = T(g0) + us.x - P.lgx0;
                    bool in = dx >= T(0);
                    if (TAB && dabs<T>(dx) < T(kEdgeTol)) {
                        range();
                        in = g0 >= glo;
                    }
                    *out = (in ? v0 : T(0)) * iq3;
                }
            }
            if (gm1 > gm0) {
                int ga = gm0 + us.s, g0 = gm0;
                T va = fs.eval(sI, spole, N, ga);
                for (; g0 + 1 < gm1; g0 += 2, ga += 2, out += 2 * N) {
                    const T vb = fs.eval(sI, spole, N, ga + 1);
                    const T vc = fs.eval(sI, spole, N, ga + 2);
                    out[0] = freq_mix<T>(va, vb, us.t) * iq3;
                    out[N] = freq_mix<T>(vb, vc, us.t) * iq3;
                    va = vc;
                }
                if (g0 < gm1) {
                    *out = freq_mix<T>(va, fs.eval(sI, spole, N, ga + 1), us.t) * iq3;
                    out += N;
                }
            }
            if (gm1 < G) {
                const T v1 = fs.eval(sI, spole, N, G - 1);
                for (int g0 = gm1; g0 < G; ++g0, out += N) {
                    const T dx = T(g0) + us.x - P.lgx1;
                    bool in = dx <= T(0);
                    if (TAB && dabs<T>(dx) < T(kEdgeTol)) {
                        range();
                        in = g0 < ghi;
                    }
                    *out = (in ? v1 : T(0)) * iq3;
                }
            }
            continue;
        }
        int hint = 0;
        for (int g0 = 0; g0 < G; ++g0) {
            const T le = tb.lc[g0] + lq;
            FreqBracket<T> fb = freq_bracket<T>(tb.lc, tb.linv, P.le0, P.leG, G, le, hint);
            if (TAB && (dabs<T>(le - P.le0) < T(kEdgeTol) || dabs<T>(le - P.leG) < T(kEdgeTol))) {
                range();  // inside or beyond the edges as the table decided
                if (g0 < glo || g0 >= ghi) fb.mode = 0;
                else if (fb.mode == 0) fb.mode = 1;  // the nearest outer group (fb.ga)
            }
            T v = 0;
            if (fb.mode == 1) {
                v = cache.get(st, sI, spole, N, fb.ga);
            } else if (fb.mode == 2) {
                T fa = cache.get(st, sI, spole, N, fb.ga);
                T fbv = cache.get(st, sI, spole, N, fb.ga + 1);
                v = freq_mix<T>(fa, fbv, fb.t);
            }
            dst[(size_t)g0 * N + k0] = v * iq3;
        }
    }
}

// comoving S0 (node-major) -> laboratory eta, chi (node-major):
// D = Gamma - u.n_k, n0 = comoving direction, eps0 = ebar_g D,
// S_lab = S0(n0, eps0)/D^3, chi_lab = chi0(eps0) D, eta_lab = chi_lab S_lab
template <class T, int TAB>
__global__ void __launch_bounds__(256, sizeof(T) == 8 ? 3 : 4) k_remap_to_lab(Prob<T> P, const T *__restrict__ S0, T *__restrict__ eta_n,
                                                      T *__restrict__ chi_n, const float4 *__restrict__ tab,
                                                      const unsigned short *__restrict__ rng)
{
    static_assert(!TAB || sizeof(T) == 4, "the remap tables are FP32");
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int G = P.G, N = P.N;
    T *sS = reinterpret_cast<T *>(smem_raw);  // [G][N] internal order
    T *spole = sS + (size_t)G * N;            // [G][2]
    T *schi = spole + 2 * G;                  // [G]
    T *slr = schi + G;                        // [G] FP32: log2(chi0[g+1]/chi0[g]) where both > 0
    const long long m = blockIdx.x;
    const long long c = P.moving[m];
    stage_node<T>(sS, S0 + m * G * N, G * N);
    for (int g = threadIdx.x; g < G; g += blockDim.x) schi[g] = P.chi0[c * G + g];
    const RemapTables<T> tb = remap_tables<T>(P, reinterpret_cast<unsigned char *>(slr + G));
    __syncthreads();
    pole_averages<T>(P, sS, tb.m2i, spole);
    for (int g = threadIdx.x; sizeof(T) == 4 && g + 1 < G; g += blockDim.x) {
        const T a = schi[g], b = schi[g + 1];
        slr[g] = (a > T(0) && b > T(0)) ? T(log2f(float(b / a))) : T(0);
    }
    __syncthreads();
    const T u[3] = {P.u[3 * c], P.u[3 * c + 1], P.u[3 * c + 2]};
    T *de = eta_n + m * G * N, *dc = chi_n + m * G * N;
    for (int k = threadIdx.x; k < N; k += blockDim.x) {
        T D;  // nu0/nu
        Stencil<T> st;
        // output groups [glo, ghi) look up source energies within the outer
        // edges (the table's FP64 decision; in place, the working precision's)
        // (read only for a lookup within kEdgeTol of an edge, as above)
        int glo = -1, ghi = -1;
        auto range = [&]() {
            if (glo < 0) {
                const unsigned r = rng[m * N + k];
                glo = (int)(r & 255u);
                ghi = (int)(r >> 8);
            }
        };
        if constexpr (TAB) {
            const float4 e = tab[m * N + k];
            D = (T)e.w;
            st = table_stencil<T>(e, P.nphi, tb.m2i);
        } else {
            T n[3] = {P.dirs[3 * k], P.dirs[3 * k + 1], P.dirs[3 * k + 2]};
            T n0[3];
            D = boost_any<T>(u, n, n0, T(1), P.fp64_boost);
            st = stencil_internal<T>(P, tb, n0);
        }
        T iD3 = T(1) / (D * D * D);
        T lD = dlog<T>(D);
        GroupCache<T> cache;
        if (sizeof(T) == 4 && P.lgu) {
            // equally spaced log centres: the constant shift s and fraction t
            // of the comoving remap above; below [gm0, gm1) chi0 is the first
            // group's, above it the last group's
            const FlatStencil<T> fs = flat_stencil<T>(st);
            const UniformShift<T> us = uniform_shift<T>(P, lD);
            const int gm0 = min(max(-us.s, 0), G), gm1 = max(min(G - 1 - us.s, G), gm0);
            T *oe = de + k, *oc = dc + k;
            if (gm0 > 0) {
                const T v0 = fs.eval(sS, spole, N, 0);
                const T chl = schi[0] * D;
                for (int g = 0; g < gm0; ++g, oe += N, oc += N) {
                    const T dx = T(g) + us.x - P.lgx0;
                    bool in = dx >= T(0);
                    if (TAB && dabs<T>(dx) < T(kEdgeTol)) {
                        range();
                        in = g >= glo;
                    }
                    *oc = chl;
                    *oe = chl * (in ? v0 : T(0)) * iD3;
                }
            }
            if (gm1 > gm0) {
                int ga = gm0 + us.s, g = gm0;
                T va = fs.eval(sS, spole, N, ga);
                // one output group: between ga and ga + 1, with V(ga + 1) = vb
                auto emit = [&](int a, T v0, T v1, T *pe, T *pc) {
                    const T c0 = schi[a], c1 = schi[a + 1];
                    const T sv = freq_mix<T>(v0, v1, us.t);
                    const T ch = (c0 > T(0) && c1 > T(0)) ? freq_mix_lr<T>(c0, slr[a], us.t)
                                                          : (T(1) - us.t) * c0 + us.t * c1;
                    const T chl = ch * D;
                    *pc = chl;
                    *pe = chl * sv * iD3;
                };
                for (; g + 1 < gm1; g += 2, ga += 2, oe += 2 * N, oc += 2 * N) {
                    const T vb = fs.eval(sS, spole, N, ga + 1);
                    const T vc = fs.eval(sS, spole, N, ga + 2);
                    emit(ga, va, vb, oe, oc);
                    emit(ga + 1, vb, vc, oe + N, oc + N);
                    va = vc;
                }
                if (g < gm1) {
                    emit(ga, va, fs.eval(sS, spole, N, ga + 1), oe, oc);
                    oe += N;
                    oc += N;
                }
            }
            if (gm1 < G) {
                const T v1 = fs.eval(sS, spole, N, G - 1);
                const T chl = schi[G - 1] * D;
                for (int g = gm1; g < G; ++g, oe += N, oc += N) {
                    const T dx = T(g) + us.x - P.lgx1;
                    bool in = dx <= T(0);
                    if (TAB && dabs<T>(dx) < T(kEdgeTol)) {
                        range();
                        in = g < ghi;
                    }
                    *oc = chl;
                    *oe = chl * (in ? v1 : T(0)) * iD3;
                }
            }
            continue;
        }
        int hint = 0;
        for (int g = 0; g < G; ++g) {
            const T le = tb.lc[g] + lD;
            FreqBracket<T> fb = freq_bracket<T>(tb.lc, tb.linv, P.le0, P.leG, G, le, hint);
            if (TAB && (dabs<T>(le - P.le0) < T(kEdgeTol) || dabs<T>(le - P.leG) < T(kEdgeTol))) {
                range();  // inside or beyond the edges as the table decided
                if (g < glo || g >= ghi) fb.mode = 0;
                else if (fb.mode == 0) fb.mode = 1;  // the nearest outer group (fb.ga)
            }
            T s = 0, ch;
            if (fb.mode == 0) {
                ch = schi[fb.ga];
            } else if (fb.mode == 1) {
                s = cache.get(st, sS, spole, N, fb.ga);
                ch = schi[fb.ga];
            } else {
                T fa = cache.get(st, sS, spole, N, fb.ga);
                T fbv = cache.get(st, sS, spole, N, fb.ga + 1);
                s = freq_mix<T>(fa, fbv, fb.t);
                ch = sizeof(T) == 4 ? chi_mix<T>(schi, slr, fb.ga, fb.t)
                                    : freq_mix<T>(schi[fb.ga], schi[fb.ga + 1], fb.t);
            }
            T chl = ch * D;
            dc[(size_t)g * N + k] = chl;
            de[(size_t)g * N + k] = chl * s * iD3;
        }
    }
}

// -------------------------------------------------------------------------
// launchers
// -------------------------------------------------------------------------
size_t remap_smem_bytes(const shd_ctx *c)
{
    // values [G][N], poles [G][2], chi0 [G], chi0 log ratios [G], tables mu,
    // lc, linv, mesh2int
    return (size_t)c->esize * ((size_t)c->G * c->N + 4 * c->G + c->nmu + 2 * c->G) + sizeof(int) * (size_t)c->N + 16;
}

size_t sh2lab_tile_smem_bytes(const shd_ctx *c)
{
    return (size_t)c->esize * ((size_t)c->NLM * 64 + (size_t)c->NLM * 128 + 128 * 65 + 64) + 64 * 4 + 64;
}

template <class T, int TC>
static cudaError_t launch_project_tile_tc(const shd_ctx *ctx, const T *I, const T *I0n, T *Ip, T *mom,
                                          cudaStream_t st)
{
    Prob<T> P = make_prob<T>(ctx);
    k_project_tile<T, TC><<<(unsigned)(ctx->ntiles * ctx->G), 128, 0, st>>>(P, I, I0n, Ip, mom);
    note_launch();
    return cudaGetLastError();
}

static int num_sms(const shd_ctx *ctx)
{
    int n = 0;
    if (cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, ctx->device) != cudaSuccess || n <= 0) n = 148;
    return n;
}

static const size_t kSmemLimit = 227 * 1024;

size_t project_persist_smem_bytes(const shd_ctx *c)
{
    return sizeof(float) * ((size_t)c->N * c->NB + 2 * 32 * 64);
}
size_t sh2lab_persist_smem_bytes(const shd_ctx *c)
{
    return sizeof(float) * ((size_t)c->NLM * c->N + (size_t)c->NLM * 64 + 128 * 65 + 64) + 64 * 4 + 64;
}

template <int TC>
static cudaError_t launch_project_persist_tc(const shd_ctx *ctx, const float *I, float *Ip, float *mom,
                                             const float *scratch, cudaStream_t st)
{
    Prob<float> P = make_prob<float>(ctx);
    size_t sm = project_persist_smem_bytes(ctx);
    cudaError_t e = cudaFuncSetAttribute(k_project_persist<TC>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    long long items = ctx->ntiles * ctx->G;
    int grid = num_sms(ctx);
    if (items < grid) grid = (int)items;
    k_project_persist<TC><<<grid, 256, sm, st>>>(P, I, scratch, Ip, mom);
    note_launch();
    return cudaGetLastError();
}

static cudaError_t launch_project_persist(const shd_ctx *ctx, const float *I, float *Ip, float *mom,
                                          const float *scratch, cudaStream_t st)
{
    switch (ctx->NB / 16) {
        case 1: return launch_project_persist_tc<1>(ctx, I, Ip, mom, scratch, st);
        case 2: return launch_project_persist_tc<2>(ctx, I, Ip, mom, scratch, st);
        case 3: return launch_project_persist_tc<3>(ctx, I, Ip, mom, scratch, st);
        case 4: return launch_project_persist_tc<4>(ctx, I, Ip, mom, scratch, st);
        case 5: return launch_project_persist_tc<5>(ctx, I, Ip, mom, scratch, st);
        case 6: return launch_project_persist_tc<6>(ctx, I, Ip, mom, scratch, st);
        case 7: return launch_project_persist_tc<7>(ctx, I, Ip, mom, scratch, st);
        case 8: return launch_project_persist_tc<8>(ctx, I, Ip, mom, scratch, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

template <class T>
static cudaError_t run_remap_to_comoving(const shd_ctx *ctx, const T *nm0, T *nm1, cudaStream_t st)
{
    Prob<T> P = make_prob<T>(ctx);
    size_t sm = remap_smem_bytes(ctx);
    const float4 *tab = sizeof(T) == 4 && ctx->rtab_valid ? (const float4 *)ctx->d_rtab[0] : nullptr;
    auto kern = (sizeof(T) == 4 && tab) ? k_remap_to_comoving<T, sizeof(T) == 4> : k_remap_to_comoving<T, 0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)ctx->nmoving, 256, sm, st>>>(P, nm0, nm1, tab, tab ? ctx->d_rrng[0] : nullptr);
    note_launch();
    return cudaGetLastError();
}

template <class T>
static cudaError_t run_remap_to_lab(const shd_ctx *ctx, const T *nm0, T *nm1, T *nm2, cudaStream_t st)
{
    Prob<T> P = make_prob<T>(ctx);
    size_t sr = remap_smem_bytes(ctx);
    const float4 *tab = sizeof(T) == 4 && ctx->rtab_valid ? (const float4 *)ctx->d_rtab[1] : nullptr;
    auto kern = (sizeof(T) == 4 && tab) ? k_remap_to_lab<T, sizeof(T) == 4> : k_remap_to_lab<T, 0>;
    cudaError_t e = cudaFuncSetAttribute(kern, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sr);
    if (e != cudaSuccess) return e;
    kern<<<(unsigned)ctx->nmoving, 256, sr, st>>>(P, nm0, nm1, nm2, tab, tab ? ctx->d_rrng[1] : nullptr);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_remap_tables_f(const shd_ctx *ctx, float4 *tc, float4 *tl, unsigned short *rc, unsigned short *rl,
                                  const double *u64, const double *dirs64, cudaStream_t st)
{
    Prob<float> P = make_prob<float>(ctx);
    const long long n = ctx->nmoving * ctx->N;
    if (n == 0) return cudaSuccess;
    k_remap_tables<<<(unsigned)((n + 255) / 256), 256, 0, st>>>(P, tc, tl, rc, rl, u64, dirs64);
    note_launch();
    return cudaGetLastError();
}

cudaError_t launch_remap_to_comoving_f(const shd_ctx *ctx, const float *nm0, float *nm1, cudaStream_t st)
{
    return run_remap_to_comoving<float>(ctx, nm0, nm1, st);
}
cudaError_t launch_remap_to_lab_f(const shd_ctx *ctx, const float *nm0, float *nm1, float *nm2, cudaStream_t st)
{
    return run_remap_to_lab<float>(ctx, nm0, nm1, nm2, st);
}

// Moving nodes first: brick transpose of I into nm0, comoving remap into
// nm1; then the projection contraction (reading nm1 for moving rows).
template <class T>
cudaError_t launch_project_nm(const shd_ctx *ctx, const T *I, T *Ip, T *mom, T *nm0, T *nm1, cudaStream_t st)
{
    Prob<T> P = make_prob<T>(ctx);
    cudaError_t e;
    if constexpr (sizeof(T) == 4) {
        // the segment kernels write the moving rows node-major themselves
        if (seg_usable(ctx)) return launch_project_seg(ctx, I, Ip, mom, nm0, nm1, st);
    }
    if (ctx->nmoving > 0) {
        k_brick_to_nodes<T><<<(unsigned)(ctx->nmtiles * ctx->G), 256, 0, st>>>(P, I, nm0);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
        if ((e = run_remap_to_comoving<T>(ctx, nm0, nm1, st)) != cudaSuccess) return e;
    }
    if constexpr (sizeof(T) == 4) {
        if (tc_usable(ctx)) return launch_project_tc(ctx, I, Ip, mom, nm1, st);
        if (project_persist_smem_bytes(ctx) <= kSmemLimit) return launch_project_persist(ctx, I, Ip, mom, nm1, st);
    }
    switch (ctx->NB / 16) {
        case 1: return launch_project_tile_tc<T, 1>(ctx, I, nm1, Ip, mom, st);
        case 2: return launch_project_tile_tc<T, 2>(ctx, I, nm1, Ip, mom, st);
        case 3: return launch_project_tile_tc<T, 3>(ctx, I, nm1, Ip, mom, st);
        case 4: return launch_project_tile_tc<T, 4>(ctx, I, nm1, Ip, mom, st);
        case 5: return launch_project_tile_tc<T, 5>(ctx, I, nm1, Ip, mom, st);
        case 6: return launch_project_tile_tc<T, 6>(ctx, I, nm1, Ip, mom, st);
        case 7: return launch_project_tile_tc<T, 7>(ctx, I, nm1, Ip, mom, st);
        case 8: return launch_project_tile_tc<T, 8>(ctx, I, nm1, Ip, mom, st);
        default: return cudaErrorInvalidConfiguration;
    }
}

template <class T>
cudaError_t launch_project(const shd_ctx *ctx, const T *I, T *Ip, T *mom, cudaStream_t st)
{
    return launch_project_nm<T>(ctx, I, Ip, mom, (T *)ctx->d_nm[0], (T *)ctx->d_nm[1], st);
}

// The contraction writes S0 of moving rows to nm0; their laboratory eta, chi
// go to nm1, nm2 and are transposed into the sweep layout.
template <class T>
cudaError_t launch_sh2lab(const shd_ctx *ctx, const T *Sp, T *eta, T *chi, cudaStream_t st, bool full_chi)
{
    Prob<T> P = make_prob<T>(ctx);
    cudaError_t e = cudaSuccess;
    T *nm0 = (T *)ctx->d_nm[0], *nm1 = (T *)ctx->d_nm[1], *nm2 = (T *)ctx->d_nm[2];
    bool done = false;
    if constexpr (sizeof(T) == 4) {
        size_t smp = sh2lab_persist_smem_bytes(ctx);
        // the segment kernels run the remap and write the moving rows themselves
        if (seg_usable(ctx)) return launch_sh2lab_seg(ctx, Sp, eta, chi, nm0, nm1, nm2, st, full_chi);
        if (tc_usable(ctx)) {
            if ((e = launch_sh2lab_tc(ctx, Sp, eta, chi, nm0, st)) != cudaSuccess) return e;
            done = true;
        } else if (smp <= kSmemLimit) {
            e = cudaFuncSetAttribute(k_sh2lab_persist, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smp);
            if (e != cudaSuccess) return e;
            long long items = ctx->ntiles * ctx->G;
            int grid = num_sms(ctx);
            if (items < grid) grid = (int)items;
            k_sh2lab_persist<<<grid, 256, smp, st>>>(P, Sp, eta, chi, nm0);
            note_launch();
            if ((e = cudaGetLastError()) != cudaSuccess) return e;
            done = true;
        }
    }
    if (!done) {
        size_t sm = sh2lab_tile_smem_bytes(ctx);
        e = cudaFuncSetAttribute(k_sh2lab_tile<T>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)sm);
        if (e != cudaSuccess) return e;
        k_sh2lab_tile<T><<<(unsigned)(ctx->ntiles * ctx->G), 256, sm, st>>>(P, Sp, eta, chi, nm0);
        note_launch();
        if ((e = cudaGetLastError()) != cudaSuccess) return e;
    }
    if (ctx->nmoving > 0) {
        if ((e = run_remap_to_lab<T>(ctx, nm0, nm1, nm2, st)) != cudaSuccess) return e;
        k_nodes_to_brick<T><<<(unsigned)(ctx->nmtiles * ctx->G), 256, 0, st>>>(P, nm1, nm2, eta, chi);
        note_launch();
        e = cudaGetLastError();
    }
    return e;
}

// Stage a1 with the moving nodes' node-major intermediates (laboratory I and
// comoving I0: 2 * nmoving * G * N reals) in caller-provided `scratch`
// instead of the context's buffers.
template <class T>
cudaError_t launch_project_scratch(const shd_ctx *ctx, const T *I, T *Ip, T *mom, T *scratch, cudaStream_t st)
{
    T *nm0 = scratch, *nm1 = scratch + (size_t)ctx->nmoving * ctx->G * ctx->N;
    return launch_project_nm<T>(ctx, I, Ip, mom, nm0, nm1, st);
}

template cudaError_t launch_project_scratch<double>(const shd_ctx *, const double *, double *, double *, double *,
                                                    cudaStream_t);
template cudaError_t launch_project_scratch<float>(const shd_ctx *, const float *, float *, float *, float *,
                                                   cudaStream_t);

template cudaError_t launch_project<double>(const shd_ctx *, const double *, double *, double *, cudaStream_t);
template cudaError_t launch_project<float>(const shd_ctx *, const float *, float *, float *, cudaStream_t);
template cudaError_t launch_sh2lab<double>(const shd_ctx *, const double *, double *, double *, cudaStream_t, bool);
template cudaError_t launch_sh2lab<float>(const shd_ctx *, const float *, float *, float *, cudaStream_t, bool);

}  // namespace shd
