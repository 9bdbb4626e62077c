// Host side of the C ABI declared in include/shdom_gb300.h: argument
// validation, set-up tables (ordinate mesh, real harmonics, sweep geometry),
// device allocation, and the order of the stages of one step (Sec. 2.2:
// lab DO -> comoving -> SH; source in SH; SH -> comoving DO -> lab; ray
// tracing).  All arithmetic of a step runs in the kernels of shd_kernels.cu.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <functional>
#include <map>
#include <mutex>
#include <vector>

#include "shd_internal.cuh"

using namespace shd;

namespace shd {
static std::atomic<unsigned long long> g_launches{0};
void note_launch() { g_launches.fetch_add(1, std::memory_order_relaxed); }
}  // namespace shd

namespace {
unsigned long long shd_launch_count_now() { return shd::g_launches.load(std::memory_order_relaxed); }
// kernels of a captured graph are counted when it is replayed, not when captured
void forget_launches(unsigned long long n) { shd::g_launches.fetch_sub(n, std::memory_order_relaxed); }
void count_launches(unsigned long long n) { shd::g_launches.fetch_add(n, std::memory_order_relaxed); }
}  // namespace

namespace {

thread_local char g_err[512] = "";

int fail(int code, const char *fmt, ...)
{
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(g_err, sizeof(g_err), fmt, ap);
    va_end(ap);
    return code;
}

int cuda_fail(cudaError_t e, const char *what)
{
    return fail(e == cudaErrorMemoryAllocation ? SHD_ERR_OOM : SHD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

#define CK(call, what)                              \
    do {                                            \
        cudaError_t e_ = (call);                    \
        if (e_ != cudaSuccess) return cuda_fail(e_, what); \
    } while (0)

bool finite_all(const double *a, size_t n, bool nonneg)
{
    for (size_t i = 0; i < n; ++i) {
        if (!std::isfinite(a[i])) return false;
        if (nonneg && a[i] < 0.0) return false;
    }
    return true;
}

// ---------------------------------------------------------------------------
// set-up tables (FP64, host)
// ---------------------------------------------------------------------------

// Gauss-Legendre nodes ascending on [-1, 1]: Newton iteration on P_n from the
// Chebyshev-like guess, weights 2 / ((1 - x^2) P_n'(x)^2).
void gauss_legendre(int n, std::vector<double> &x, std::vector<double> &w)
{
    x.assign(n, 0.0);
    w.assign(n, 0.0);
    for (int i = 0; i < n; ++i) {
        double z = std::cos(kPi * (n - i - 0.25) / (n + 0.5));  // ascending guess
        double pn = 0, dpn = 0;
        for (int it = 0; it < 100; ++it) {
            double pm = 1.0, pc = z;  // P_0, P_1
            for (int j = 1; j < n; ++j) {
                double pnext = ((2 * j + 1) * z * pc - j * pm) / (j + 1);
                pm = pc;
                pc = pnext;
            }
            if (n == 0) pc = 1.0;
            pn = pc;                                   // P_n
            dpn = n * (pm - z * pc) / (1.0 - z * z);  // P_n' from P_{n-1}
            if (n == 1) dpn = 1.0;
            double dz = pn / dpn;
            z -= dz;
            if (std::fabs(dz) <= 1e-16 * std::fmax(1.0, std::fabs(z))) break;
        }
        double pm = 1.0, pc = z;
        for (int j = 1; j < n; ++j) {
            double pnext = ((2 * j + 1) * z * pc - j * pm) / (j + 1);
            pm = pc;
            pc = pnext;
        }
        dpn = (n == 1) ? 1.0 : n * (pm - z * pc) / (1.0 - z * z);
        x[i] = z;
        w[i] = 2.0 / ((1.0 - z * z) * dpn * dpn);
    }
}

// Real orthonormal harmonics Y_p(mu, phi), p = l*l + l + m (Sec. 2.3): the
// associated Legendre functions without the (-1)^m phase by the standard
// upward recurrences in l, times sqrt((2 - d_m0)(2l+1)/4pi (l-m)!/(l+m)!)
// and cos(m phi) (m > 0) / sin(|m| phi) (m < 0).
void real_harmonics(int L, double mu, double phi, double *Y)
{
    double sth = std::sqrt(std::fmax(0.0, (1.0 - mu) * (1.0 + mu)));
    double pmm = 1.0;  // P_m^m
    for (int m = 0; m <= L; ++m) {
        if (m > 0) pmm *= (2.0 * m - 1.0) * sth;
        double cm = std::cos(m * phi), sm = std::sin(m * phi);
        double p_lm2 = 0.0, p_lm1 = pmm;
        for (int l = m; l <= L; ++l) {
            double plm;
            if (l == m) {
                plm = pmm;
            } else if (l == m + 1) {
                plm = (2.0 * m + 1.0) * mu * pmm;
            } else {
                plm = ((2.0 * l - 1.0) * mu * p_lm1 - (l + m - 1.0) * p_lm2) / (double)(l - m);
            }
            if (l > m) { p_lm2 = p_lm1; p_lm1 = plm; }
            double ratio = 1.0;  // (l-m)!/(l+m)!
            for (int q = l - m + 1; q <= l + m; ++q) ratio /= (double)q;
            double nrm = std::sqrt((m ? 2.0 : 1.0) * (2.0 * l + 1.0) / (4.0 * kPi) * ratio);
            if (m == 0) {
                Y[l * l + l] = nrm * plm;
            } else {
                Y[l * l + l + m] = nrm * plm * cm;
                Y[l * l + l - m] = nrm * plm * sm;
            }
        }
    }
}

template <class T>
void *to_device_vec(const std::vector<double> &v, long long &bytes, cudaError_t &err)
{
    std::vector<T> tmp(v.begin(), v.end());
    void *p = nullptr;
    err = cudaMalloc(&p, tmp.size() * sizeof(T) + 16);
    if (err != cudaSuccess) return nullptr;
    bytes += (long long)(tmp.size() * sizeof(T));
    err = cudaMemcpy(p, tmp.data(), tmp.size() * sizeof(T), cudaMemcpyHostToDevice);
    return p;
}

void dfree(void *&p)
{
    if (p) cudaFree(p);
    p = nullptr;
}

void free_all(shd_ctx *c)
{
    void **ptrs[] = {&c->d_ord, &c->d_W, &c->d_dirs, &c->d_Y, &c->d_mu, (void **)&c->d_edges, (void **)&c->d_centre,
                     &c->d_alpha0, &c->d_ne, &c->d_u, &c->d_emis0, &c->d_chi0, &c->d_K, &c->d_sigma_out, &c->d_bc,
                     &c->d_I, &c->d_eta, &c->d_chi, &c->d_Ip, &c->d_Sp, &c->d_Sprev, &c->d_mom,
                     (void **)&c->d_sums, (void **)&c->d_partial, (void **)&c->d_stage,
                     &c->d_tiles, (void **)&c->d_moving, (void **)&c->d_mflag, &c->d_Bproj,
                     (void **)&c->d_midx, (void **)&c->d_mtiles, &c->d_nm[0], &c->d_nm[1], &c->d_nm[2],
                     &c->d_lc, &c->d_linv, &c->d_tc_Bh, &c->d_tc_Bl, &c->d_tc_Yh, &c->d_tc_Yl,
                     (void **)&c->d_int2mesh, (void **)&c->d_mesh2int,
                     &c->d_chi0L, (void **)&c->d_mbits, &c->d_seg[0], &c->d_seg[1], &c->d_tcs_Bh[0], &c->d_tcs_Bh[1], &c->d_tcs_Bl[0],
                     &c->d_tcs_Bl[1], &c->d_tcs_Yh[0], &c->d_tcs_Yh[1], &c->d_tcs_Yl[0], &c->d_tcs_Yl[1],
                     (void **)&c->d_tc_err, &c->d_rtab[0], &c->d_rtab[1], (void **)&c->d_rrng[0],
                     (void **)&c->d_rrng[1], &c->d_dirs64, &c->d_fstage, &c->d_fcheck,
                     &c->d_ng[0], &c->d_ng[1], &c->d_ng[2], (void **)&c->d_ngpart, &c->d_rk[0], &c->d_rk[1],
                     &c->d_rk[2], (void **)&c->d_sums_save, &c->d_tcK, (void **)&c->d_thb,
                     (void **)&c->d_thperm, &c->d_thw, &c->d_thK, &c->d_thso, (void **)&c->d_thchunk,
                     (void **)&c->d_chi_dirty};
    for (void **p : ptrs) dfree(*p);
    c->bytes = 0;
    c->rtab_n = 0;
    c->rtab_valid = false;
    c->fstage_n = 0;
}

bool is_fp64(const shd_ctx *c) { return c->precision == SHD_FP64; }

int ctx_check(shd_ctx *c)
{
    if (!c) return fail(SHD_ERR_ARG, "null context");
    cudaError_t e = cudaSetDevice(c->device);
    if (e != cudaSuccess) return cuda_fail(e, "cudaSetDevice");
    return SHD_OK;
}

int dalloc(shd_ctx *c, void **p, size_t bytes, const char *what)
{
    dfree(*p);
    cudaError_t e = cudaMalloc(p, bytes ? bytes : 16);
    if (e != cudaSuccess) {
        *p = nullptr;
        return fail(SHD_ERR_OOM, "cudaMalloc %s (%zu bytes): %s", what, bytes, cudaGetErrorString(e));
    }
    c->bytes += (long long)bytes;
    return SHD_OK;
}

// drop everything that depends on the problem sizes
void drop_sized(shd_ctx *c)
{
    c->chi_rest_state = 2;
    c->sweep_C = c->sweep_NT = 0;  // the sweep schedule depends on the sizes
    c->sweep_ntune = 0;
    void **ptrs[] = {&c->d_alpha0, &c->d_ne, &c->d_u, &c->d_emis0, &c->d_chi0, &c->d_K, &c->d_sigma_out, &c->d_bc,
                     &c->d_I, &c->d_eta, &c->d_chi, &c->d_Ip, &c->d_Sp, &c->d_Sprev, &c->d_mom,
                     (void **)&c->d_partial, (void **)&c->d_stage,
                     &c->d_tiles, (void **)&c->d_moving, (void **)&c->d_mflag,
                     (void **)&c->d_midx, (void **)&c->d_mtiles, &c->d_nm[0], &c->d_nm[1], &c->d_nm[2],
                     &c->d_rtab[0], &c->d_rtab[1], (void **)&c->d_rrng[0], (void **)&c->d_rrng[1], &c->d_fstage,
                     &c->d_ng[0], &c->d_ng[1], &c->d_ng[2],
                     &c->d_rk[0], &c->d_rk[1], &c->d_rk[2], &c->d_tcK, (void **)&c->d_thb,
                     (void **)&c->d_thperm, &c->d_thw, &c->d_thK, &c->d_thso, (void **)&c->d_thchunk};
    for (void **p : ptrs) dfree(*p);
    c->ntiles = 0;
    c->nmoving = 0;
    c->rtab_n = 0;
    c->rtab_valid = false;
    c->fstage_n = 0;
    c->have_fields = c->have_scat = c->have_state = false;
    c->have_theta = false;
    c->h_theta.clear();
    c->nthchunk = 0;
    c->bc_mode = SHD_BC_VACUUM;
    c->sprev_valid = false;
}

// Sweep geometry of every ordinate: the face crossed first (largest
// |n_a|/h_a, ties to the lowest axis), the path length s = h_d/|n_d| back to
// it, and the in-plane offsets s |n_e| / h_e of the upwind point.
void build_geometry(shd_ctx *c)
{
    c->h_ord.assign(c->N, Ordinate());
    for (int k = 0; k < c->N; ++k) {
        Ordinate &o = c->h_ord[k];
        for (int a = 0; a < 3; ++a) o.n[a] = c->h_dirs[3 * k + a];
        o.W = c->h_W[k];
        o.ring = c->h_int2mesh[k] / c->nphi;
        o.phi = c->h_int2mesh[k] % c->nphi;
        if (!c->have_grid) continue;
        int d = 0;
        double best = std::fabs(o.n[0]) / c->h[0];
        for (int a = 1; a < 3; ++a) {
            double v = std::fabs(o.n[a]) / c->h[a];
            if (v > best) { best = v; d = a; }
        }
        o.d = d;
        if (d == 2) { o.e1 = 1; o.e2 = 0; }
        else if (d == 1) { o.e1 = 2; o.e2 = 0; }
        else { o.e1 = 2; o.e2 = 1; }
        o.s = c->h[d] / std::fabs(o.n[d]);
        o.fr1 = o.s * std::fabs(o.n[o.e1]) / c->h[o.e1];
        o.fr2 = o.s * std::fabs(o.n[o.e2]) / c->h[o.e2];
        auto sgn = [](double v) { return (v > 0.0) - (v < 0.0); };
        o.sd = sgn(o.n[d]);
        o.s1 = sgn(o.n[o.e1]);
        o.s2 = sgn(o.n[o.e2]);
    }
}

// Projection matrix of stage a1, [N][NB]: W_k Y_p(n_k) for p < NLM, then the
// ten moment weights W_k {1, n_x, n_y, n_z, n_x^2, n_y^2, n_z^2, n_x n_y,
// n_x n_z, n_y n_z} / (4 pi), then zero padding to NB = 16 ceil((NLM+10)/16).
std::vector<double> projection_matrix(const shd_ctx *c)
{
    int NB = c->NB;
    std::vector<double> B((size_t)c->N * NB, 0.0);
    for (int k = 0; k < c->N; ++k) {
        double W = c->h_W[k];
        const double *n = &c->h_dirs[3 * k];
        double *row = &B[(size_t)k * NB];
        for (int p = 0; p < c->NLM; ++p) row[p] = W * c->h_Y[(size_t)k * c->NLM + p];
        double f[10] = {1.0, n[0], n[1], n[2], n[0] * n[0], n[1] * n[1], n[2] * n[2], n[0] * n[1], n[0] * n[2],
                        n[1] * n[2]};
        for (int m = 0; m < 10; ++m) row[c->NLM + m] = W * f[m] / (4.0 * kPi);
    }
    return B;
}

// BF16 round-to-nearest-even of a float (finite inputs).
uint16_t bf16_rne(float f)
{
    uint32_t u;
    std::memcpy(&u, &f, 4);
    u += 0x7FFFu + ((u >> 16) & 1u);
    return (uint16_t)(u >> 16);
}
double bf16_val(uint16_t h)
{
    uint32_t u = (uint32_t)h << 16;
    float f;
    std::memcpy(&f, &u, 4);
    return (double)f;
}

int canon_offset(int r, int k, int K) { return (((r >> 3) * (K >> 3) + (k >> 3)) << 6) + ((r & 7) << 3) + (k & 7); }

// BF16 hi / lo device copies (canonical K-major layout) of the rows [0, nr)
// x columns [0, nk) of at(r, k), zero-padded to rows x K.
static void split_upload(shd_ctx *c, void **dh, void **dl, int rows, int K, const std::function<double(int, int)> &at,
                         int nr, int nk, int &rc)
{
    std::vector<uint16_t> h((size_t)rows * K, 0), l(h.size(), 0);
    for (int r = 0; r < nr; ++r)
        for (int k = 0; k < nk; ++k) {
            const double x = at(r, k);
            const uint16_t hh = bf16_rne((float)x);
            const int o = canon_offset(r, k, K);
            h[o] = hh;
            l[o] = bf16_rne((float)(x - bf16_val(hh)));
        }
    if ((rc = dalloc(c, dh, h.size() * 2, "tc segment operand"))) return;
    if ((rc = dalloc(c, dl, l.size() * 2, "tc segment operand"))) return;
    cudaError_t e = cudaMemcpy(*dh, h.data(), h.size() * 2, cudaMemcpyHostToDevice);
    if (e == cudaSuccess) e = cudaMemcpy(*dl, l.data(), l.size() * 2, cudaMemcpyHostToDevice);
    if (e != cudaSuccess) rc = cuda_fail(e, "tc segment operand");
}

// Segment tiling and per-group operands of the mixed path (needs the grid:
// the classes follow the axis each ordinate crosses first).
int upload_seg_operands(shd_ctx *c, const std::vector<double> &Bp)
{
    for (int grp = 0; grp < 2; ++grp) {
        dfree(c->d_seg[grp]); dfree(c->d_tcs_Bh[grp]); dfree(c->d_tcs_Bl[grp]);
        dfree(c->d_tcs_Yh[grp]); dfree(c->d_tcs_Yl[grp]);
        c->nseg[grp] = 0;
        c->tcs_Kp[grp] = c->tcs_nchunk[grp] = 0;
    }
    c->seg_ready = false;
    if (c->precision != SHD_MIXED || !c->have_grid) return SHD_OK;
    auto pow2_box = [](int n) {
        int b = 4;
        while (b < n && b < 128) b *= 2;
        return b;
    };
    int rc = SHD_OK;
    for (int grp = 0; grp < 2; ++grp) {
        // the group's classes: {map index, first internal ordinate, count}
        int cls[2][3];
        int ncls = 0;
        if (grp == 0) {
            if (c->nZ > 0) { cls[ncls][0] = 0; cls[ncls][1] = 0; cls[ncls][2] = c->nZ; ++ncls; }
            if (c->nA > c->nZ) { cls[ncls][0] = 1; cls[ncls][1] = c->nZ; cls[ncls][2] = c->nA - c->nZ; ++ncls; }
        } else if (c->N > c->nA) {
            cls[ncls][0] = 0; cls[ncls][1] = c->nA; cls[ncls][2] = c->N - c->nA; ++ncls;
        }
        if (ncls == 0) continue;
        std::vector<int> slot;  // internal ordinate of each slot, -1 at padding
        int nch = 0;
        for (int q = 0; q < ncls; ++q)
            for (int k0 = 0; k0 < cls[q][2]; k0 += 32) {
                if (nch == 16) return SHD_OK;  // more than 512 slots: the brick kernels take over
                c->tcs_chunk[grp][nch][0] = cls[q][0];
                c->tcs_chunk[grp][nch][1] = k0;
                c->tcs_chunk[grp][nch][2] = cls[q][1];
                c->tcs_chunk[grp][nch][3] = cls[q][2];
                ++nch;
                for (int i = 0; i < 32; ++i) slot.push_back(k0 + i < cls[q][2] ? cls[q][1] + k0 + i : -1);
            }
        c->tcs_nchunk[grp] = nch;
        c->tcs_Kp[grp] = 32 * nch;
        split_upload(c, &c->d_tcs_Bh[grp], &c->d_tcs_Bl[grp], c->NB, c->tcs_Kp[grp],
                     [&](int j, int s) { return slot[s] < 0 ? 0.0 : Bp[(size_t)slot[s] * c->NB + j]; }, c->NB,
                     c->tcs_Kp[grp], rc);
        if (rc) return rc;
        split_upload(c, &c->d_tcs_Yh[grp], &c->d_tcs_Yl[grp], c->tcs_Kp[grp], c->tc_Kq,
                     [&](int s, int p) { return slot[s] < 0 ? 0.0 : c->h_Y[(size_t)slot[s] * c->NLM + p]; },
                     c->tcs_Kp[grp], c->NLM, rc);
        if (rc) return rc;
        // tiles: group 0 boxes of (x, y) at each z, group 1 of (y, z) at each x
        const int na = grp ? c->ny : c->nx, nbb = grp ? c->nz : c->ny, nplane = grp ? c->nx : c->nz;
        const int bw = pow2_box(na), bh = 128 / bw;
        c->seg_bw[grp] = bw;
        std::vector<int> seg;
        for (int pl = 0; pl < nplane; ++pl)
            for (int b0 = 0; b0 < nbb; b0 += bh)
                for (int a0 = 0; a0 < na; a0 += bw) {
                    seg.push_back(pl);
                    seg.push_back(a0);
                    seg.push_back(b0);
                    seg.push_back(0);
                }
        c->nseg[grp] = (long long)seg.size() / 4;
        if ((rc = dalloc(c, &c->d_seg[grp], seg.size() * sizeof(int), "segments"))) return rc;
        CK(cudaMemcpy(c->d_seg[grp], seg.data(), seg.size() * sizeof(int), cudaMemcpyHostToDevice), "segments");
    }
    c->seg_ready = true;
    return SHD_OK;
}

// Tensor-core operands of the mixed path: a value x is stored as BF16
// hi = bf16(x) and lo = bf16(x - hi), in the canonical K-major layout.
int upload_tc_operands(shd_ctx *c, const std::vector<double> &Bp)
{
    dfree(c->d_tc_Bh); dfree(c->d_tc_Bl); dfree(c->d_tc_Yh); dfree(c->d_tc_Yl);
    if (c->precision != SHD_MIXED) return SHD_OK;
    auto up = [](int v, int m) { return (v + m - 1) / m * m; };
    c->tc_Kp = up(c->N, 32);
    c->tc_Np = up(c->N, 32);
    c->tc_Kq = up(c->NLM, 16);
    std::vector<uint16_t> bh((size_t)c->NB * c->tc_Kp, 0), bl(bh.size(), 0);
    for (int k = 0; k < c->N; ++k)
        for (int j = 0; j < c->NB; ++j) {
            double x = Bp[(size_t)k * c->NB + j];
            uint16_t h = bf16_rne((float)x);
            uint16_t l = bf16_rne((float)(x - bf16_val(h)));
            int o = canon_offset(j, k, c->tc_Kp);
            bh[o] = h;
            bl[o] = l;
        }
    std::vector<uint16_t> yh((size_t)c->tc_Np * c->tc_Kq, 0), yl(yh.size(), 0);
    for (int k = 0; k < c->N; ++k)
        for (int p = 0; p < c->NLM; ++p) {
            double x = c->h_Y[(size_t)k * c->NLM + p];
            uint16_t h = bf16_rne((float)x);
            uint16_t l = bf16_rne((float)(x - bf16_val(h)));
            int o = canon_offset(k, p, c->tc_Kq);
            yh[o] = h;
            yl[o] = l;
        }
    int rc;
    if ((rc = dalloc(c, &c->d_tc_Bh, bh.size() * 2, "tc Bh"))) return rc;
    if ((rc = dalloc(c, &c->d_tc_Bl, bl.size() * 2, "tc Bl"))) return rc;
    if ((rc = dalloc(c, &c->d_tc_Yh, yh.size() * 2, "tc Yh"))) return rc;
    if ((rc = dalloc(c, &c->d_tc_Yl, yl.size() * 2, "tc Yl"))) return rc;
    CK(cudaMemcpy(c->d_tc_Bh, bh.data(), bh.size() * 2, cudaMemcpyHostToDevice), "tc Bh");
    CK(cudaMemcpy(c->d_tc_Bl, bl.data(), bl.size() * 2, cudaMemcpyHostToDevice), "tc Bl");
    CK(cudaMemcpy(c->d_tc_Yh, yh.data(), yh.size() * 2, cudaMemcpyHostToDevice), "tc Yh");
    CK(cudaMemcpy(c->d_tc_Yl, yl.data(), yl.size() * 2, cudaMemcpyHostToDevice), "tc Yl");
    return upload_seg_operands(c, Bp);
}

// Internal ordinate order: grouped by the axis each ordinate crosses first
// (z, then y, then x; mesh order within a group), so that the ordinates of
// a group share one sweep layout.  Without a grid yet: mesh order.
void order_ordinates(shd_ctx *c)
{
    const int N = c->N;
    std::vector<int> cls(N, 2);
    if (c->have_grid) {
        for (int k = 0; k < N; ++k) {
            const double *n = &c->h_dirs_mesh[3 * k];
            int d = 0;
            double best = std::fabs(n[0]) / c->h[0];
            for (int a = 1; a < 3; ++a) {
                double v = std::fabs(n[a]) / c->h[a];
                if (v > best) { best = v; d = a; }
            }
            cls[k] = d;
        }
    }
    c->h_int2mesh.clear();
    for (int want : {2, 1, 0})
        for (int k = 0; k < N; ++k)
            if (cls[k] == want) c->h_int2mesh.push_back(k);
    c->nA = 0;
    c->nZ = 0;
    for (int k = 0; k < N; ++k) {
        c->nA += cls[k] != 0;
        c->nZ += cls[k] == 2;
    }
    c->h_mesh2int.assign(N, 0);
    for (int i = 0; i < N; ++i) c->h_mesh2int[c->h_int2mesh[i]] = i;
    c->h_dirs.assign(3 * (size_t)N, 0.0);
    c->h_W.assign(N, 0.0);
    c->h_Y.assign((size_t)N * c->NLM, 0.0);
    for (int i = 0; i < N; ++i) {
        const int k = c->h_int2mesh[i];
        for (int q = 0; q < 3; ++q) c->h_dirs[3 * i + q] = c->h_dirs_mesh[3 * k + q];
        c->h_W[i] = c->h_W_mesh[k];
        for (int p = 0; p < c->NLM; ++p) c->h_Y[(size_t)i * c->NLM + p] = c->h_Y_mesh[(size_t)k * c->NLM + p];
    }
}

int upload_angles(shd_ctx *c)
{
    dfree(c->d_ord); dfree(c->d_W); dfree(c->d_dirs); dfree(c->d_Y); dfree(c->d_mu); dfree(c->d_Bproj);
    dfree(c->d_dirs64);
    dfree((void *&)c->d_int2mesh); dfree((void *&)c->d_mesh2int);
    order_ordinates(c);
    build_geometry(c);
    {
        int rc;
        if ((rc = dalloc(c, (void **)&c->d_int2mesh, sizeof(int) * c->N, "int2mesh"))) return rc;
        if ((rc = dalloc(c, (void **)&c->d_mesh2int, sizeof(int) * c->N, "mesh2int"))) return rc;
        CK(cudaMemcpy(c->d_int2mesh, c->h_int2mesh.data(), sizeof(int) * c->N, cudaMemcpyHostToDevice), "int2mesh");
        CK(cudaMemcpy(c->d_mesh2int, c->h_mesh2int.data(), sizeof(int) * c->N, cudaMemcpyHostToDevice), "mesh2int");
    }
    c->NB = 16 * ((c->NLM + 10 + 15) / 16);
    std::vector<double> Bp = projection_matrix(c);
    cudaError_t e;
    CK(cudaMalloc(&c->d_ord, sizeof(Ordinate) * c->N), "cudaMalloc ordinates");
    CK(cudaMemcpy(c->d_ord, c->h_ord.data(), sizeof(Ordinate) * c->N, cudaMemcpyHostToDevice), "copy ordinates");
    if (is_fp64(c)) {
        c->d_W = to_device_vec<double>(c->h_W, c->bytes, e); CK(e, "W");
        c->d_dirs = to_device_vec<double>(c->h_dirs, c->bytes, e); CK(e, "dirs");
        c->d_Y = to_device_vec<double>(c->h_Y, c->bytes, e); CK(e, "Y");
        c->d_mu = to_device_vec<double>(c->h_mu, c->bytes, e); CK(e, "mu");
        c->d_Bproj = to_device_vec<double>(Bp, c->bytes, e); CK(e, "Bproj");
    } else {
        c->d_W = to_device_vec<float>(c->h_W, c->bytes, e); CK(e, "W");
        c->d_dirs = to_device_vec<float>(c->h_dirs, c->bytes, e); CK(e, "dirs");
        c->d_Y = to_device_vec<float>(c->h_Y, c->bytes, e); CK(e, "Y");
        c->d_mu = to_device_vec<float>(c->h_mu, c->bytes, e); CK(e, "mu");
        c->d_Bproj = to_device_vec<float>(Bp, c->bytes, e); CK(e, "Bproj");
    }
    // FP64 directions for the remap tables' edge decisions
    c->d_dirs64 = to_device_vec<double>(c->h_dirs, c->bytes, e); CK(e, "dirs (FP64)");
    return upload_tc_operands(c, Bp);
}

bool sized(const shd_ctx *c) { return c->have_grid && c->have_angles && c->have_groups; }

// Allocate the state-sized buffers once grid, angles and groups are known.
int ensure_buffers(shd_ctx *c)
{
    if (!sized(c)) return fail(SHD_ERR_STATE, "grid, angles and groups must be set first");
    if (c->d_I) return SHD_OK;
    size_t es = c->esize;
    size_t nDO = (size_t)c->Nc * c->G * c->N, nSH = (size_t)c->Nc * c->G * c->NLM, nCG = (size_t)c->Nc * c->G;
    int rc;
    // (+16 bytes: the FP32 sweep copies a plane's aligned cover, which may
    // reach up to 12 bytes past the last plane)
    if ((rc = dalloc(c, &c->d_I, nDO * es + 16, "I"))) return rc;
    if ((rc = dalloc(c, &c->d_eta, nDO * es + 16, "eta_lab"))) return rc;
    if ((rc = dalloc(c, &c->d_chi, nDO * es + 16, "chi_lab"))) return rc;
    if ((rc = dalloc(c, &c->d_Ip, nSH * es, "I_lm"))) return rc;
    if ((rc = dalloc(c, &c->d_Sp, nSH * es, "S_lm"))) return rc;
    if ((rc = dalloc(c, &c->d_Sprev, nSH * es, "S_lm prev"))) return rc;
    if ((rc = dalloc(c, &c->d_mom, nCG * 10 * es, "moments"))) return rc;
    if ((rc = dalloc(c, &c->d_alpha0, nCG * es, "alpha0"))) return rc;
    if ((rc = dalloc(c, &c->d_emis0, nCG * es, "emis0"))) return rc;
    if ((rc = dalloc(c, &c->d_chi0, nCG * es, "chi0"))) return rc;
    if ((rc = dalloc(c, &c->d_chi0L, 3 * nCG * es, "chi0 layouts"))) return rc;
    if ((rc = dalloc(c, (void **)&c->d_chi_dirty, sizeof(int), "chi0 change word"))) return rc;
    CK(cudaMemset(c->d_chi_dirty, 0, sizeof(int)), "chi0 change word");
    c->chi_rest_state = 2;
    if ((rc = dalloc(c, &c->d_ne, (size_t)c->Nc * es, "ne"))) return rc;
    if ((rc = dalloc(c, &c->d_u, (size_t)c->Nc * 3 * es, "u"))) return rc;
    c->n_partial = 8 * 152;
    if ((rc = dalloc(c, (void **)&c->d_partial, sizeof(double) * 4 * c->n_partial, "partials"))) return rc;
    size_t per_node = (size_t)c->G * c->N;
    size_t want = per_node > ((size_t)1 << 24) ? per_node : ((size_t)1 << 24);  // >= 16 Mi doubles or one node
    size_t cap = (size_t)c->Nc * per_node;
    if (want > cap) want = cap;
    if ((rc = dalloc(c, (void **)&c->d_stage, sizeof(double) * want, "staging"))) return rc;
    c->stage_elems = want;
    CK(cudaMemsetAsync(c->d_Sprev, 0, nSH * es, c->stream), "memset");
    return SHD_OK;
}

// Make `waiter` wait for the work enqueued so far on `producer`.
int stream_after(cudaStream_t waiter, cudaStream_t producer)
{
    if (waiter == producer) return SHD_OK;
    cudaEvent_t ev;
    CK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming), "event");
    cudaError_t e = cudaEventRecord(ev, producer);
    if (e == cudaSuccess) e = cudaStreamWaitEvent(waiter, ev, 0);
    cudaEventDestroy(ev);
    if (e != cudaSuccess) return cuda_fail(e, "stream ordering");
    return SHD_OK;
}

// Node bricks of the transform kernels and the list of moving nodes (u != 0),
// brick by brick so that a brick's remap CTAs run side by side.
int build_tiles(shd_ctx *c, const double *u)
{
    c->chi_rest_state = 2;  // nodes that stop moving need chi0 in chi_lab again
    dfree(c->d_tiles); dfree((void *&)c->d_moving); dfree((void *&)c->d_mflag); dfree((void *&)c->d_mbits);
    dfree((void *&)c->d_midx); dfree((void *&)c->d_mtiles);
    for (int i = 0; i < 3; ++i) dfree(c->d_nm[i]);
    int tx = (c->nx + 7) / 8, ty = (c->ny + 7) / 8;
    std::vector<TileInfo> tiles;
    tiles.reserve((size_t)tx * ty * c->nz);
    std::vector<long long> moving;
    std::vector<unsigned char> mflag((size_t)c->Nc, 0);
    std::vector<int> midx((size_t)c->Nc, -1), mtiles;
    for (int z = 0; z < c->nz; ++z)
        for (int by = 0; by < ty; ++by)
            for (int bx = 0; bx < tx; ++bx) {
                TileInfo t{8 * bx, 8 * by, z, 0};
                for (int r = 0; r < 64; ++r) {
                    int ix = t.x0 + (r & 7), iy = t.y0 + (r >> 3);
                    if (ix >= c->nx || iy >= c->ny) continue;
                    long long node = ((long long)z * c->ny + iy) * c->nx + ix;
                    const double *un = u + 3 * node;
                    if (un[0] != 0.0 || un[1] != 0.0 || un[2] != 0.0) {
                        t.flags |= 1;
                        mflag[node] = 1;
                        midx[node] = (int)moving.size();
                        moving.push_back(node);
                    }
                }
                if (t.flags & 1) mtiles.push_back((int)tiles.size());
                tiles.push_back(t);
            }
    c->ntiles = (long long)tiles.size();
    c->nmoving = (long long)moving.size();
    {
        // moving 4-node pieces of every plane of the three sweep layouts
        const int dims[3] = {c->nx, c->ny, c->nz};
        int npc = 0, nwin = 0;
        for (int d = 0; d < 3; ++d) {
            const int e1 = d == 0 ? 2 : (d == 1 ? 2 : 1), e2 = d == 0 ? 1 : 0;  // layout (d, e1, e2)
            const int plane = dims[e1] * dims[e2];
            npc = std::max(npc, (plane + 3) / 4);
            nwin = std::max(nwin, (dims[d] + 63) / 64);
        }
        std::vector<unsigned long long> bits((size_t)3 * nwin * npc, 0ull);
        for (long long node = 0; node < c->Nc; ++node) {
            if (!mflag[node]) continue;
            const int ix = (int)(node % c->nx), iy = (int)((node / c->nx) % c->ny), iz = (int)(node / ((long long)c->nx * c->ny));
            for (int d = 0; d < 3; ++d) {
                const long long o = perm_offset(d, ix, iy, iz, c->nx, c->ny, c->nz);
                const int plane = d == 2 ? c->nx * c->ny : (d == 1 ? c->nx * c->nz : c->ny * c->nz);
                const int id = (int)(o / plane), j = (int)(o % plane);
                bits[((size_t)d * nwin + id / 64) * npc + j / 4] |= 1ull << (id % 64);
            }
        }
        c->mbits_npc = npc;
        c->mbits_nwin = nwin;
        int rc0;
        if ((rc0 = dalloc(c, (void **)&c->d_mbits, bits.size() * sizeof(unsigned long long), "moving pieces")))
            return rc0;
        CK(cudaMemcpy(c->d_mbits, bits.data(), bits.size() * sizeof(unsigned long long), cudaMemcpyHostToDevice),
           "moving pieces");
    }
    int rc;
    if ((rc = dalloc(c, &c->d_tiles, sizeof(TileInfo) * tiles.size(), "tiles"))) return rc;
    CK(cudaMemcpy(c->d_tiles, tiles.data(), sizeof(TileInfo) * tiles.size(), cudaMemcpyHostToDevice), "tiles");
    if ((rc = dalloc(c, (void **)&c->d_mflag, mflag.size(), "mflag"))) return rc;
    CK(cudaMemcpy(c->d_mflag, mflag.data(), mflag.size(), cudaMemcpyHostToDevice), "mflag");
    if ((rc = dalloc(c, (void **)&c->d_midx, sizeof(int) * midx.size(), "midx"))) return rc;
    CK(cudaMemcpy(c->d_midx, midx.data(), sizeof(int) * midx.size(), cudaMemcpyHostToDevice), "midx");
    c->nmtiles = (long long)mtiles.size();
    if (c->nmoving > 0) {
        if ((rc = dalloc(c, (void **)&c->d_moving, sizeof(long long) * moving.size(), "moving"))) return rc;
        CK(cudaMemcpy(c->d_moving, moving.data(), sizeof(long long) * moving.size(), cudaMemcpyHostToDevice), "moving");
        if ((rc = dalloc(c, (void **)&c->d_mtiles, sizeof(int) * mtiles.size(), "mtiles"))) return rc;
        CK(cudaMemcpy(c->d_mtiles, mtiles.data(), sizeof(int) * mtiles.size(), cudaMemcpyHostToDevice), "mtiles");
        size_t nNM = (size_t)c->nmoving * c->G * c->N;
        for (int i = 0; i < 3; ++i)
            if ((rc = dalloc(c, &c->d_nm[i], nNM * c->esize, "remap scratch"))) return rc;
    }
    return SHD_OK;
}

template <class T>
int set_state_impl(shd_ctx *c, const double *src, bool host, cudaStream_t st, T *dst)
{
    size_t per_node = (size_t)c->G * c->N;
    long long chunk = (long long)(c->stage_elems / per_node);
    if (chunk < 1) chunk = 1;
    for (long long c0 = 0; c0 < c->Nc; c0 += chunk) {
        long long nc = c->Nc - c0 < chunk ? c->Nc - c0 : chunk;
        const double *s = src + (size_t)c0 * per_node;
        if (host) {
            CK(cudaMemcpyAsync(c->d_stage, s, sizeof(double) * nc * per_node, cudaMemcpyHostToDevice, st), "H2D state");
            s = c->d_stage;
        }
        CK(launch_canon_to_do<T>(c, s, dst, c0, nc, st), "canon_to_do");
    }
    return SHD_OK;
}

template <class T>
int get_state_impl(shd_ctx *c, const T *src, double *dst, bool host, cudaStream_t st)
{
    size_t per_node = (size_t)c->G * c->N;
    long long chunk = (long long)(c->stage_elems / per_node);
    if (chunk < 1) chunk = 1;
    for (long long c0 = 0; c0 < c->Nc; c0 += chunk) {
        long long nc = c->Nc - c0 < chunk ? c->Nc - c0 : chunk;
        double *d = dst + (size_t)c0 * per_node;
        if (host) {
            CK(launch_do_to_canon<T>(c, src, c->d_stage, c0, nc, st), "do_to_canon");
            CK(cudaMemcpyAsync(d, c->d_stage, sizeof(double) * nc * per_node, cudaMemcpyDeviceToHost, st), "D2H state");
            CK(cudaStreamSynchronize(st), "sync");
        } else {
            CK(launch_do_to_canon<T>(c, src, d, c0, nc, st), "do_to_canon");
        }
    }
    return SHD_OK;
}

// Upload a host FP64 array of n reals into a device real array (via staging).
template <class T>
int upload_reals(shd_ctx *c, const double *h, void *dst, size_t n)
{
    size_t off = 0;
    while (off < n) {
        size_t m = n - off < c->stage_elems ? n - off : c->stage_elems;
        CK(cudaMemcpyAsync(c->d_stage, h + off, sizeof(double) * m, cudaMemcpyHostToDevice, c->stream), "H2D");
        CK(launch_convert<T>(c->d_stage, (T *)dst + off, (long long)m, c->stream), "convert");
        off += m;
    }
    return SHD_OK;
}

template <class T>
int download_reals(shd_ctx *c, const void *src, double *h, size_t n)
{
    size_t off = 0;
    while (off < n) {
        size_t m = n - off < c->stage_elems ? n - off : c->stage_elems;
        CK(launch_convert_back<T>((const T *)src + off, c->d_stage, (long long)m, c->stream), "convert");
        CK(cudaMemcpyAsync(h + off, c->d_stage, sizeof(double) * m, cudaMemcpyDeviceToHost, c->stream), "D2H");
        CK(cudaStreamSynchronize(c->stream), "sync");
        off += m;
    }
    return SHD_OK;
}

// A tensor-core kernel that gave up on a bounded wait leaves a flag behind;
// the next synchronous call reports it (and clears it).
int check_device_flags(shd_ctx *c)
{
    int flag = 0;
    CK(cudaMemcpyAsync(&flag, c->d_tc_err, sizeof(int), cudaMemcpyDeviceToHost, c->stream), "read flag");
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (flag) {
        cudaMemsetAsync(c->d_tc_err, 0, sizeof(int), c->stream);
        return fail(SHD_ERR_TIMEOUT, "a tensor-core kernel gave up (a bounded wait ran out)");
    }
    return SHD_OK;
}

int ready_for_step(shd_ctx *c)
{
    if (!sized(c)) return fail(SHD_ERR_STATE, "grid, angles and groups must be set");
    if (!c->have_fields) return fail(SHD_ERR_STATE, "fields not set");
    if (!c->have_scat) return fail(SHD_ERR_STATE, "scattering not set");
    if (c->scat_kind == SHD_SCAT_KN_THERMAL && !c->have_theta)
        return fail(SHD_ERR_STATE, "the thermal Compton kernel needs the electron temperatures (theta_e)");
    size_t limit = 227 * 1024;
    if (remap_smem_bytes(c) > limit)
        return fail(SHD_ERR_ARG, "groups x ordinates too large for the remap kernels (%zu bytes shared memory)",
                    remap_smem_bytes(c));
    if (sh2lab_tile_smem_bytes(c) > limit)
        return fail(SHD_ERR_ARG, "too many harmonics for the sh2lab kernel (%zu bytes shared memory)",
                    sh2lab_tile_smem_bytes(c));
    if (sweep_smem_bytes(c) > limit) return fail(SHD_ERR_ARG, "grid planes too large for the sweep kernel");
    if (c->integrator == SHD_SC_BEZIER && !sweep_bez_usable(c))
        return fail(SHD_ERR_ARG, "grid planes too large for the Bezier sweep (at most 4096 nodes, %zu bytes "
                                 "of shared memory a node pair in this precision)", 2 * 6 * c->esize);
    return SHD_OK;
}

}  // namespace

namespace shd {
// ready_for_step for the other translation units (its message: shd_last_error)
int check_ready(shd_ctx *c) { return ready_for_step(c); }
}  // namespace shd

namespace {

struct FieldCheck {
    unsigned int bad, moving_changed, u_changed, pad;
    unsigned long long max_alpha, max_ne, max_uu;
};

// One pass over the fields as given (FP64, device staging): which of them
// hold a non-finite (or, for alpha0, ne, emis0, negative) value (bits 0-3:
// alpha0, ne, u, emis0), the maxima of alpha0, ne and |u|^2 (bit patterns of
// non-negative doubles, which order like the integers), whether a node's
// moving flag differs from prev_mflag and whether u, rounded to the working
// precision, differs from prev_u (the previous fields; null on the first call).
template <class T>
__global__ void __launch_bounds__(256) k_check_fields(const double *__restrict__ alpha0, const double *__restrict__ ne,
                                                      const double *__restrict__ u, const double *__restrict__ emis0,
                                                      long long nCG, long long Nc,
                                                      const unsigned char *__restrict__ prev_mflag,
                                                      const T *__restrict__ prev_u, FieldCheck *out)
{
    unsigned bad = 0, mch = 0, uch = 0;
    double ma = 0.0, mn = 0.0, mu = 0.0;
    const long long stride = (long long)gridDim.x * blockDim.x;
    const long long i0 = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    for (long long i = i0; i < nCG; i += stride) {
        const double a = alpha0[i], e = emis0[i];
        if (!(isfinite(a) && a >= 0.0)) bad |= 1u;
        else ma = fmax(ma, a);
        if (!(isfinite(e) && e >= 0.0)) bad |= 8u;
    }
    for (long long i = i0; i < Nc; i += stride) {
        const double n = ne[i];
        if (!(isfinite(n) && n >= 0.0)) bad |= 2u;
        else mn = fmax(mn, n);
        const double u0 = u[3 * i], u1 = u[3 * i + 1], u2 = u[3 * i + 2];
        if (!(isfinite(u0) && isfinite(u1) && isfinite(u2))) {
            bad |= 4u;
            continue;
        }
        mu = fmax(mu, u0 * u0 + u1 * u1 + u2 * u2);
        const unsigned char mv = (u0 != 0.0 || u1 != 0.0 || u2 != 0.0) ? 1 : 0;
        if (prev_mflag && mv != prev_mflag[i]) mch = 1u;
        if (prev_u && ((T)u0 != prev_u[3 * i] || (T)u1 != prev_u[3 * i + 1] || (T)u2 != prev_u[3 * i + 2])) uch = 1u;
    }
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) {
        bad |= __shfl_xor_sync(0xffffffffu, bad, o);
        mch |= __shfl_xor_sync(0xffffffffu, mch, o);
        uch |= __shfl_xor_sync(0xffffffffu, uch, o);
        ma = fmax(ma, __shfl_xor_sync(0xffffffffu, ma, o));
        mn = fmax(mn, __shfl_xor_sync(0xffffffffu, mn, o));
        mu = fmax(mu, __shfl_xor_sync(0xffffffffu, mu, o));
    }
    if ((threadIdx.x & 31) == 0) {
        if (bad) atomicOr(&out->bad, bad);
        if (mch) atomicOr(&out->moving_changed, mch);
        if (uch) atomicOr(&out->u_changed, uch);
        atomicMax(&out->max_alpha, (unsigned long long)__double_as_longlong(ma));
        atomicMax(&out->max_ne, (unsigned long long)__double_as_longlong(mn));
        atomicMax(&out->max_uu, (unsigned long long)__double_as_longlong(mu));
    }
}

template <class T>
cudaError_t check_fields(shd_ctx *c, const double *alpha0, const double *ne, const double *u, const double *emis0,
                         const unsigned char *prev_mflag, const T *prev_u, FieldCheck &fc)
{
    FieldCheck *d = (FieldCheck *)c->d_fcheck;
    cudaError_t e = cudaMemsetAsync(d, 0, sizeof(FieldCheck), c->stream);
    if (e != cudaSuccess) return e;
    int sms = 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, c->device) != cudaSuccess || sms <= 0) sms = 148;
    k_check_fields<T><<<4 * sms, 256, 0, c->stream>>>(alpha0, ne, u, emis0, (long long)c->Nc * c->G, c->Nc,
                                                       prev_mflag, prev_u, d);
    note_launch();
    if ((e = cudaGetLastError()) != cudaSuccess) return e;
    if ((e = cudaMemcpyAsync(&fc, d, sizeof(FieldCheck), cudaMemcpyDeviceToHost, c->stream)) != cudaSuccess) return e;
    return cudaStreamSynchronize(c->stream);
}

// The FP32 remap tables of the moving nodes, built on the library's stream
// when the flow or the angles changed since the last build; stream st (if
// any) then waits for them, else the host does.  Without them the remap
// kernels compute the boosts and stencils in place.
int ensure_remap_tables(shd_ctx *c, cudaStream_t st)
{
    // (the entries pack the ring index in 10 bits, the group ranges in 8)
    if (is_fp64(c) || c->rtab_valid || c->nmoving == 0 || !c->have_fields || !c->have_angles || c->nmu > 1024 ||
        c->G > 255 || !c->d_fstage || !c->fstage_u_current || !c->d_dirs64)
        return SHD_OK;
    const size_t n = (size_t)c->nmoving * c->N;
    int rc;
    if (n != c->rtab_n || !c->d_rtab[0] || !c->d_rtab[1] || !c->d_rrng[0] || !c->d_rrng[1]) {
        c->rtab_n = 0;
        for (int i = 0; i < 2; ++i) {
            if ((rc = dalloc(c, &c->d_rtab[i], n * sizeof(float4), "remap tables"))) return rc;
            if ((rc = dalloc(c, (void **)&c->d_rrng[i], n * sizeof(unsigned short), "remap group ranges"))) return rc;
        }
        c->rtab_n = n;
    }
    // the flow as last given (FP64), still in the field staging area
    const size_t nCG = (size_t)c->Nc * c->G;
    const double *u64 = (const double *)c->d_fstage + 2 * nCG + (size_t)c->Nc;
    CK(launch_remap_tables_f(c, (float4 *)c->d_rtab[0], (float4 *)c->d_rtab[1], c->d_rrng[0], c->d_rrng[1], u64,
                             (const double *)c->d_dirs64, c->stream),
       "remap tables");
    if (st) {
        if ((rc = stream_after(st, c->stream))) return rc;
    } else {
        CK(cudaStreamSynchronize(c->stream), "remap tables");
    }
    c->rtab_valid = true;
    return SHD_OK;
}

// The segment transform (MIXED) stores chi_lab only where a node moves.  The
// sweep reads chi at rest from the chi0 layout table where it can (aligned
// rows, c0L); elsewhere -- other sweep kernels, or rows not a multiple of 4
// nodes, where a 4-node piece may straddle a moving and a resting row -- it
// reads chi_lab, whose entries at rest then come from one fill with chi0.
template <class T>
bool rest_chi_kept(const shd_ctx *c)
{
    if constexpr (sizeof(T) == 4)
        return c->precision == SHD_MIXED && seg_usable(c) && c->d_chi0L && c->d_chi_dirty;
    return false;
}
template <class T>
bool rest_chi_read(const shd_ctx *c)
{
    return rest_chi_kept<T>(c) && (!sweep_uses_chi0L<T>(c) || seg_manual(c));
}

// The fill of chi_lab at rest on st where the sweep reads it and chi0 or the
// moving set changed (kept outside captured steps: run_steps and the batch
// call this before capturing; with chi0 unchanged it exits at once).
template <class T>
int ensure_chi_rest(shd_ctx *c, cudaStream_t st)
{
    if (c->chi_rest_state == 0 || !rest_chi_read<T>(c)) return SHD_OK;
    CK(launch_chi_rest_fill<T>(c, (T *)c->d_chi, st, c->chi_rest_state == 2), "chi at rest");
    c->chi_rest_state = 0;
    return SHD_OK;
}

// The kernels of one step on stream st (timing events around the stages when
// ev is given); S_lm / S_prev are not swapped here.
template <class T>
int step_once(shd_ctx *c, cudaStream_t st, cudaEvent_t *ev, const std::function<int()> *after_source = nullptr)
{
    const bool tm = ev != nullptr;
    if (tm) CK(cudaEventRecord(ev[0], st), "event");
    CK(launch_project<T>(c, (const T *)c->d_I, (T *)c->d_Ip, (T *)c->d_mom, st), "project");
    if (tm) CK(cudaEventRecord(ev[1], st), "event");
    if (source_sums_usable<T>(c)) {
        // a2 with the a5 partials in the same pass; the sums stage is the final reduction
        CK(launch_source_sums<T>(c, (const T *)c->d_Ip, (T *)c->d_Sp, (const T *)c->d_mom, (const T *)c->d_Sprev,
                                 c->sprev_valid, st),
           "source and sums");
        if (tm) CK(cudaEventRecord(ev[2], st), "event");
        if (tm) CK(cudaEventRecord(ev[3], st), "event");
    } else {
        CK(launch_source<T>(c, (const T *)c->d_Ip, (T *)c->d_Sp, st), "source");
        if (tm) CK(cudaEventRecord(ev[2], st), "event");
        CK(launch_sums<T>(c, (const T *)c->d_mom, (const T *)c->d_Sp, (const T *)c->d_Sprev, c->sprev_valid, st),
           "sums");
        if (tm) CK(cudaEventRecord(ev[3], st), "event");
    }
    // a caller's step between the source and its transform (Ng extrapolation)
    if (after_source && *after_source) {
        int rc = (*after_source)();
        if (rc) return rc;
    }
    // the sweep takes chi at nodes at rest from the chi0 layouts (c0L), or
    // from chi_lab, where the segment transform leaves chi0 of the one-time
    // fill: either way a3 stores chi only where a node moves
    const bool c0L = sweep_uses_chi0L<T>(c);
    bool full_chi = !c0L;
    if (rest_chi_kept<T>(c)) {
        if (int rc = ensure_chi_rest<T>(c, st)) return rc;  // where the sweep reads chi_lab at rest
        full_chi = false;
    }
    CK(launch_sh2lab<T>(c, (const T *)c->d_Sp, (T *)c->d_eta, (T *)c->d_chi, st, full_chi), "sh2lab");
    if (tm) CK(cudaEventRecord(ev[4], st), "event");
    if (!c->skip_sweep)  // (a batch sweeps every problem of it in one launch)
        CK(launch_sweep<T>(c, (T *)c->d_I, (const T *)c->d_eta, (const T *)c->d_chi, st, c0L), "sweep");
    if (tm) CK(cudaEventRecord(ev[5], st), "event");
    return SHD_OK;
}

// The Runge-Kutta arrays (allocated before any capture needs them).
int ensure_rk_buffers(shd_ctx *c)
{
    if (c->time_scheme != SHD_TIME_RK4) return SHD_OK;
    const size_t n = (size_t)c->Nc * c->G * c->N;
    int rc;
    for (int i = 0; i < 3; ++i)
        if (!c->d_rk[i] && (rc = dalloc(c, &c->d_rk[i], n * c->esize, "Runge-Kutta arrays"))) return rc;
    if (!c->d_sums_save && (rc = dalloc(c, (void **)&c->d_sums_save, 2 * sizeof(double), "saved sums"))) return rc;
    return SHD_OK;
}

// The next per-stage timing slot of a recorded sub-solve, or null.
cudaEvent_t *timing_slot(shd_ctx *c)
{
    if (!(c->timing.on && c->timing.count < Timing::kCap)) return nullptr;
    return &c->timing.pool[(size_t)c->timing.count++ * (Timing::kStages + 1)];
}

// One time step on stream st.  SHD_TIME_EULER: one source iteration with
// the backward-Euler time term (Sec. 2.1, eq:time).  SHD_TIME_RK4: App. A,
// eq:rk4th: four sub-solves from I(t) with time steps dt/6, dt/3, dt/3, dt/6
// (kappa = 1/(c dt) scaled by 6, 3, 3, 6), each one source iteration; after
// sub-solve i with increment dI_i = result - input, the next input is
// I(t) + 3 dI_1, I(t) + 3/2 dI_2, I(t) + 3 dI_3, and the new state is
// I(t) + dI_1 + dI_2 + dI_3 + dI_4.  The sums report the energy and photon
// number of I(t) (first sub-solve) and the source change of the last.
// S_lm / S_prev are swapped between sub-solves here, and after the step by
// the caller.
template <class T>
int step_full(shd_ctx *c, cudaStream_t st)
{
    if (c->time_scheme != SHD_TIME_RK4) return step_once<T>(c, st, timing_slot(c));
    const long long n = (long long)c->Nc * c->G * c->N;
    T *I = (T *)c->d_I, *A = (T *)c->d_rk[0], *B = (T *)c->d_rk[1], *acc = (T *)c->d_rk[2];
    if (!A || !B || !acc || !c->d_sums_save) return fail(SHD_ERR_STATE, "Runge-Kutta arrays missing");
    CK(cudaMemcpyAsync(A, I, n * sizeof(T), cudaMemcpyDeviceToDevice, st), "RK copy");
    CK(cudaMemcpyAsync(B, I, n * sizeof(T), cudaMemcpyDeviceToDevice, st), "RK copy");
    static const double frac[4] = {1.0 / 6.0, 1.0 / 3.0, 1.0 / 3.0, 1.0 / 6.0};
    static const double cnext[4] = {3.0, 1.5, 3.0, 0.0};
    const double kap = c->kappa;
    int rc = SHD_OK;
    for (int i = 0; i < 4 && rc == SHD_OK; ++i) {
        c->kappa = kap / frac[i];
        rc = step_once<T>(c, st, timing_slot(c));
        if (rc) break;
        if (i == 0) {
            cudaError_t e = cudaMemcpyAsync(c->d_sums_save, c->d_sums, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st);
            if (e != cudaSuccess) { rc = cuda_fail(e, "save sums"); break; }
        }
        cudaError_t e = launch_rk_stage<T>(I, A, B, acc, n, cnext[i], i == 0, i == 3, st);
        if (e != cudaSuccess) { rc = cuda_fail(e, "Runge-Kutta stage"); break; }
        if (i < 3) {
            std::swap(c->d_Sp, c->d_Sprev);
            c->sprev_valid = true;
        }
    }
    c->kappa = kap;
    if (rc) return rc;
    CK(cudaMemcpyAsync(c->d_sums, c->d_sums_save, 2 * sizeof(double), cudaMemcpyDeviceToDevice, st), "restore sums");
    return SHD_OK;
}

void drop_graphs(shd_ctx *c)
{
    for (int i = 0; i < 2; ++i) {
        if (c->gexec[i]) cudaGraphExecDestroy(c->gexec[i]);
        if (c->graph[i]) cudaGraphDestroy(c->graph[i]);
        if (c->graph_ns[i]) cudaGraphDestroy(c->graph_ns[i]);
        c->gexec[i] = nullptr;
        c->graph[i] = nullptr;
        c->graph_sp[i] = nullptr;
        c->graph_kernels[i] = 0;
        c->graph_ns[i] = nullptr;
        c->graph_ns_sp[i] = nullptr;
        c->graph_ns_kernels[i] = 0;
    }
    c->graph_gen++;
}

// The step without its sweep (a backward-Euler step), as the context stands,
// captured for a batch that sweeps its problems together; *slot is its
// graph_ns slot, -1 when it cannot be captured.
template <class T>
int capture_presweep(shd_ctx *c, int *slot)
{
    *slot = -1;
    for (int i = 0; i < 2; ++i)
        if (c->graph_ns[i] && c->graph_ns_sp[i] == c->d_Sp) {
            *slot = i;
            return SHD_OK;
        }
    if (c->time_scheme != SHD_TIME_EULER) return SHD_OK;
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
    int rt = ensure_remap_tables(c, nullptr);
    if (rt) return rt;
    const int i = c->graph_ns[0] ? 1 : 0;
    if (c->graph_ns[i]) {
        cudaGraphDestroy(c->graph_ns[i]);
        c->graph_ns[i] = nullptr;
    }
    const unsigned long long n0 = shd_launch_count_now();
    void *sp0 = c->d_Sp, *sprev0 = c->d_Sprev;
    const bool valid0 = c->sprev_valid;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    c->skip_sweep = true;
    const int rc = step_once<T>(c, c->cap_stream, nullptr);
    c->skip_sweep = false;
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
    c->d_Sp = sp0;
    c->d_Sprev = sprev0;
    c->sprev_valid = valid0;
    const unsigned long long n = shd_launch_count_now() - n0;
    forget_launches(n);
    cudaGetLastError();
    if (rc != SHD_OK || ee != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        return SHD_OK;  // this problem's batch step keeps its own sweep
    }
    c->graph_ns[i] = graph;
    c->graph_ns_sp[i] = c->d_Sp;
    c->graph_ns_kernels[i] = n;
    c->graph_gen++;
    *slot = i;
    return SHD_OK;
}

// Capture one step, as the context stands, into graph slot i.
template <class T>
int capture_step(shd_ctx *c, int i)
{
    if (!c->cap_stream) CK(cudaStreamCreateWithFlags(&c->cap_stream, cudaStreamNonBlocking), "capture stream");
    int rt = ensure_remap_tables(c, nullptr);  // built outside the graph, read in place by every replay
    if (rt) return rt;
    if ((rt = ensure_rk_buffers(c))) return rt;
    const unsigned long long n0 = shd_launch_count_now();
    void *sp0 = c->d_Sp, *sprev0 = c->d_Sprev;
    const bool valid0 = c->sprev_valid;
    CK(cudaStreamBeginCapture(c->cap_stream, cudaStreamCaptureModeThreadLocal), "begin capture");
    const int rc = step_full<T>(c, c->cap_stream);
    cudaGraph_t graph = nullptr;
    const cudaError_t ee = cudaStreamEndCapture(c->cap_stream, &graph);
    // nothing ran: the buffers the step swapped while it was captured are
    // put back as they stand before the step
    c->d_Sp = sp0;
    c->d_Sprev = sprev0;
    c->sprev_valid = valid0;
    const unsigned long long n = shd_launch_count_now() - n0;
    forget_launches(n);  // captured, not launched
    cudaGetLastError();
    if (rc != SHD_OK || ee != cudaSuccess || !graph) {
        if (graph) cudaGraphDestroy(graph);
        c->graphs_off = true;
        return SHD_OK;  // the caller launches directly
    }
    cudaGraphExec_t exec = nullptr;
    const cudaError_t ei = cudaGraphInstantiate(&exec, graph, 0);
    if (ei != cudaSuccess) {
        cudaGraphDestroy(graph);
        cudaGetLastError();
        c->graphs_off = true;
        return SHD_OK;
    }
    c->graph[i] = graph;  // kept: a batch step embeds it as a child graph
    c->gexec[i] = exec;
    c->graph_sp[i] = c->d_Sp;
    c->graph_kernels[i] = n;
    c->graph_gen++;
    return SHD_OK;
}

// The graph slot of the context's next step (capturing it if needed), or -1
// when that step runs as direct launches.
template <class T>
int graph_slot(shd_ctx *c, int &slot)
{
    slot = -1;
    const bool tm = c->timing.on && c->timing.count < Timing::kCap;
    if (tm || !c->sprev_valid || c->graphs_off) return SHD_OK;
    int i = c->graph_sp[0] == c->d_Sp ? 0 : (c->graph_sp[1] == c->d_Sp ? 1 : -1);
    if (i < 0) {
        i = c->gexec[0] ? 1 : 0;
        int rc = capture_step<T>(c, i);
        if (rc) return rc;
        if (c->graphs_off) return SHD_OK;
    }
    slot = i;
    return SHD_OK;
}

// The timed choice of the FP32 sweep schedule, shared by every context of
// the same shape in the process: a problem whose shape was timed before
// takes that choice (and its timing record) instead of timing again.
struct SchedKey {
    int device, nx, ny, nz, G, N, ncls[3], bits;
    bool operator<(const SchedKey &o) const { return std::memcmp(this, &o, sizeof(SchedKey)) < 0; }
};
struct SchedChoice {
    int C, NT, ntune;
    float tune[16][3];
};
std::mutex g_sched_mu;
std::map<SchedKey, SchedChoice> g_sched_cache;

bool sched_key(const shd_ctx *c, SchedKey &k)
{
    if (c->precision == SHD_FP64 || c->integrator != SHD_SC_LINEAR || c->sweep_force_C > 0) return false;
    std::memset(&k, 0, sizeof(k));
    k.device = c->device;
    k.nx = c->nx; k.ny = c->ny; k.nz = c->nz;
    k.G = c->G; k.N = c->N;
    for (const Ordinate &o : c->h_ord) k.ncls[o.d]++;
    k.bits = sweep_uses_chi0L<float>(c) ? 1 : 0;
    return true;
}

void sched_cache_take(shd_ctx *c)
{
    SchedKey k;
    if (c->sweep_C > 0 || !sched_key(c, k)) return;
    std::lock_guard<std::mutex> lock(g_sched_mu);
    auto it = g_sched_cache.find(k);
    if (it == g_sched_cache.end() || !sweep_schedule_valid(c, it->second.C, it->second.NT)) return;
    c->sweep_C = it->second.C;
    c->sweep_NT = it->second.NT;
    c->sweep_ntune = it->second.ntune;
    std::memcpy(c->sweep_tune, it->second.tune, sizeof(c->sweep_tune));
}

void sched_cache_keep(const shd_ctx *c)
{
    SchedKey k;
    if (c->sweep_C <= 0 || c->sweep_ntune <= 0 || !sched_key(c, k)) return;
    SchedChoice v;
    v.C = c->sweep_C;
    v.NT = c->sweep_NT;
    v.ntune = c->sweep_ntune;
    std::memcpy(v.tune, c->sweep_tune, sizeof(v.tune));
    std::lock_guard<std::mutex> lock(g_sched_mu);
    g_sched_cache.emplace(k, v);
}

template <class T>
int run_steps(shd_ctx *c, int nsteps, cudaStream_t st, bool graphs = false,
              const std::function<int()> *after_source = nullptr)
{
    if constexpr (sizeof(T) == 4) sched_cache_take(c);
    if (int rc = ensure_remap_tables(c, st)) return rc;
    if (int rc = ensure_rk_buffers(c)) return rc;
    if (int rc = ensure_chi_rest<T>(c, st)) return rc;  // before any capture
    for (int s = 0; s < nsteps; ++s) {
        // a replay of the captured step: a step with S_prev, no timing events
        if (graphs) {
            int i;
            int rc = graph_slot<T>(c, i);
            if (rc) return rc;
            if (i >= 0) {
                CK(cudaGraphLaunch(c->gexec[i], st), "graph launch");
                count_launches(c->graph_kernels[i]);
                std::swap(c->d_Sp, c->d_Sprev);
                continue;
            }
        }
        int rc = after_source ? step_once<T>(c, st, timing_slot(c), after_source) : step_full<T>(c, st);
        if (rc) return rc;
        std::swap(c->d_Sp, c->d_Sprev);
        c->sprev_valid = true;
        if constexpr (sizeof(T) == 4) sched_cache_keep(c);
    }
    return SHD_OK;
}

}  // namespace

// ===========================================================================
// C ABI
// ===========================================================================

extern "C" {

unsigned long long shd_launch_count(void) { return shd_launch_count_now(); }

const char *shd_last_error(void) { return g_err; }

int shd_create(shd_ctx **out, int device, int precision)
{
    if (!out) return fail(SHD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (precision != SHD_FP64 && precision != SHD_FP32 && precision != SHD_MIXED)
        return fail(SHD_ERR_ARG, "unknown precision %d", precision);
    int ndev = 0;
    cudaError_t e = cudaGetDeviceCount(&ndev);
    if (e != cudaSuccess) return cuda_fail(e, "cudaGetDeviceCount");
    if (device < 0 || device >= ndev) return fail(SHD_ERR_ARG, "device %d out of range (%d devices)", device, ndev);
    CK(cudaSetDevice(device), "cudaSetDevice");
    shd_ctx *c = new (std::nothrow) shd_ctx();
    if (!c) return fail(SHD_ERR_OOM, "host allocation");
    c->device = device;
    c->precision = precision;
    c->esize = precision == SHD_FP64 ? 8 : 4;
    e = cudaStreamCreateWithFlags(&c->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) { delete c; return cuda_fail(e, "cudaStreamCreate"); }
    e = cudaMalloc(&c->d_sums, sizeof(double) * 4);
    if (e != cudaSuccess) { cudaStreamDestroy(c->stream); delete c; return cuda_fail(e, "cudaMalloc"); }
    cudaMemset(c->d_sums, 0, sizeof(double) * 4);
    e = cudaMalloc(&c->d_tc_err, sizeof(int));
    if (e != cudaSuccess) { cudaFree(c->d_sums); cudaStreamDestroy(c->stream); delete c; return cuda_fail(e, "cudaMalloc"); }
    cudaMemset(c->d_tc_err, 0, sizeof(int));
    *out = c;
    g_err[0] = 0;
    return SHD_OK;
}

void shd_destroy(shd_ctx *c)
{
    if (!c) return;
    cudaSetDevice(c->device);
    if (c->stream) cudaStreamSynchronize(c->stream);
    cudaDeviceSynchronize();  // graph replays may run on callers' streams
    drop_graphs(c);
    free_all(c);
    for (cudaEvent_t e : c->timing.pool) cudaEventDestroy(e);
    if (c->cap_stream) cudaStreamDestroy(c->cap_stream);
    if (c->stream) cudaStreamDestroy(c->stream);
    delete c;
}

int shd_set_grid(shd_ctx *c, int nx, int ny, int nz, double lx, double ly, double lz)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    drop_graphs(c);  // the captured step holds the old parameters
    if (nx < 2 || ny < 2 || nz < 2) return fail(SHD_ERR_ARG, "every grid dimension must be >= 2");
    if (!(lx > 0 && ly > 0 && lz > 0) || !std::isfinite(lx) || !std::isfinite(ly) || !std::isfinite(lz))
        return fail(SHD_ERR_ARG, "box lengths must be positive and finite");
    long long Nc = (long long)nx * ny * nz;
    if (Nc > (1LL << 31)) return fail(SHD_ERR_ARG, "too many nodes");
    drop_sized(c);
    c->nx = nx; c->ny = ny; c->nz = nz;
    c->lx = lx; c->ly = ly; c->lz = lz;
    c->h[0] = lx / (nx - 1); c->h[1] = ly / (ny - 1); c->h[2] = lz / (nz - 1);
    c->Nc = Nc;
    c->have_grid = true;
    if (c->have_angles) return upload_angles(c);
    return SHD_OK;
}

int shd_set_angles(shd_ctx *c, int L, int n_mu, int n_phi)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    drop_graphs(c);  // the captured step holds the old parameters
    if (L < 0 || L > 9) return fail(SHD_ERR_ARG, "L must be in [0, 9]");
    if (n_mu < L + 1 || n_phi < 2 * L + 1) return fail(SHD_ERR_ARG, "need n_mu >= L+1 and n_phi >= 2L+1");
    if (n_mu < 1 || n_phi < 1 || (long long)n_mu * n_phi > 4096) return fail(SHD_ERR_ARG, "n_mu*n_phi must be in [1, 4096]");
    drop_sized(c);
    c->L = L; c->nmu = n_mu; c->nphi = n_phi;
    c->N = n_mu * n_phi;
    c->NLM = (L + 1) * (L + 1);
    gauss_legendre(n_mu, c->h_mu, c->h_wmu);
    c->h_dirs_mesh.assign(3 * c->N, 0.0);
    c->h_W_mesh.assign(c->N, 0.0);
    c->h_Y_mesh.assign((size_t)c->N * c->NLM, 0.0);
    for (int a = 0; a < n_mu; ++a) {
        double sth = std::sqrt((1.0 - c->h_mu[a]) * (1.0 + c->h_mu[a]));
        for (int b = 0; b < n_phi; ++b) {
            int k = a * n_phi + b;
            double phi = 2.0 * kPi * b / n_phi;
            double n[3] = {sth * std::cos(phi), sth * std::sin(phi), c->h_mu[a]};
            for (int q = 0; q < 3; ++q) c->h_dirs_mesh[3 * k + q] = std::fabs(n[q]) < 1e-12 ? 0.0 : n[q];
            c->h_W_mesh[k] = c->h_wmu[a] * (2.0 * kPi / n_phi);
            real_harmonics(L, c->h_mu[a], phi, &c->h_Y_mesh[(size_t)k * c->NLM]);
        }
    }
    c->have_angles = true;
    return upload_angles(c);
}

int shd_set_groups(shd_ctx *c, int G, const double *edges)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    drop_graphs(c);  // the captured step holds the old parameters
    if (G < 1 || G > 256 || !edges) return fail(SHD_ERR_ARG, "need 1 <= G <= 256 and edges");
    for (int g = 0; g <= G; ++g)
        if (!std::isfinite(edges[g]) || edges[g] <= 0.0 || (g > 0 && !(edges[g] > edges[g - 1])))
            return fail(SHD_ERR_ARG, "edges must be positive, finite and strictly ascending");
    drop_sized(c);
    c->G = G;
    c->h_edges.assign(edges, edges + G + 1);
    c->h_centre.assign(G, 0.0);
    for (int g = 0; g < G; ++g) c->h_centre[g] = std::sqrt(edges[g] * edges[g + 1]);
    dfree((void *&)c->d_edges);
    dfree((void *&)c->d_centre);
    cudaError_t e;
    c->d_edges = (double *)to_device_vec<double>(c->h_edges, c->bytes, e); CK(e, "edges");
    c->d_centre = (double *)to_device_vec<double>(c->h_centre, c->bytes, e); CK(e, "centres");
    // log-energy tables of the frame remaps: log centres and inverse spacings
    std::vector<double> lc(G), linv(G, 0.0);
    for (int g = 0; g < G; ++g) lc[g] = std::log(c->h_centre[g]);
    for (int g = 0; g + 1 < G; ++g) linv[g] = 1.0 / (lc[g + 1] - lc[g]);
    // centres equally spaced in log energy (geometric groups)?
    c->lg_uniform = G >= 2;
    c->lg_dl = G >= 2 ? (lc[G - 1] - lc[0]) / (G - 1) : 1.0;
    c->lg_c0 = lc[0];
    for (int g = 0; g + 1 < G && c->lg_uniform; ++g)
        if (std::fabs((lc[g + 1] - lc[g]) - c->lg_dl) > 1e-9 * std::fabs(c->lg_dl)) c->lg_uniform = false;
    dfree(c->d_lc);
    dfree(c->d_linv);
    if (is_fp64(c)) {
        c->d_lc = to_device_vec<double>(lc, c->bytes, e); CK(e, "log centres");
        c->d_linv = to_device_vec<double>(linv, c->bytes, e); CK(e, "log spacings");
    } else {
        c->d_lc = to_device_vec<float>(lc, c->bytes, e); CK(e, "log centres");
        c->d_linv = to_device_vec<float>(linv, c->bytes, e); CK(e, "log spacings");
    }
    c->have_groups = true;
    return SHD_OK;
}

// Node temperatures: the bracket of each node on the temperature grid and
// the weight of the upper table (FP64 on the host, linear in log10(theta),
// clamped into the grid), and the nodes grouped by bracket in chunks of at
// most kThermalChunk for the source pass.
int set_theta(shd_ctx *c, const double *theta)
{
    const size_t Nc = (size_t)c->Nc;
    for (size_t i = 0; i < Nc; ++i)
        if (!std::isfinite(theta[i]) || theta[i] < 0.0) return fail(SHD_ERR_NAN, "theta_e must be finite and >= 0");
    const bool same = c->have_theta && c->h_theta.size() == Nc &&
                      std::equal(theta, theta + Nc, c->h_theta.begin());
    if (same) return SHD_OK;
    drop_graphs(c);  // the source pass's chunks are baked into a captured step
    c->h_theta.assign(theta, theta + Nc);
    std::vector<int> b(Nc), cnt(kThermalN, 0);
    std::vector<double> w(Nc);
    for (size_t i = 0; i < Nc; ++i) {
        double x = theta[i] > 0.0 ? (std::log10(theta[i]) - kThermalLg0) / kThermalDlg : 0.0;
        x = std::min(std::max(x, 0.0), (double)(kThermalN - 1));
        int i0 = std::min((int)std::floor(x), kThermalN - 2);
        b[i] = i0;
        w[i] = x - i0;
        cnt[i0]++;
    }
    std::vector<int> start(kThermalN, 0), perm(Nc);
    for (int k = 1; k < kThermalN; ++k) start[k] = start[k - 1] + cnt[k - 1];
    std::vector<int> pos = start;
    for (size_t i = 0; i < Nc; ++i) perm[pos[b[i]]++] = (int)i;
    std::vector<int4> chunks;
    for (int k = 0; k < kThermalN; ++k)
        for (int j = 0; j < cnt[k]; j += kThermalChunk)
            chunks.push_back(make_int4(start[k] + j, std::min(kThermalChunk, cnt[k] - j), k, 0));
    int rc;
    if ((rc = dalloc(c, (void **)&c->d_thb, Nc * sizeof(int), "theta brackets"))) return rc;
    if ((rc = dalloc(c, (void **)&c->d_thperm, Nc * sizeof(int), "theta order"))) return rc;
    if ((rc = dalloc(c, &c->d_thw, Nc * c->esize, "theta weights"))) return rc;
    if ((rc = dalloc(c, (void **)&c->d_thchunk, chunks.size() * sizeof(int4), "theta chunks"))) return rc;
    CK(cudaMemcpy(c->d_thb, b.data(), Nc * sizeof(int), cudaMemcpyHostToDevice), "theta brackets");
    CK(cudaMemcpy(c->d_thperm, perm.data(), Nc * sizeof(int), cudaMemcpyHostToDevice), "theta order");
    CK(cudaMemcpy(c->d_thchunk, chunks.data(), chunks.size() * sizeof(int4), cudaMemcpyHostToDevice), "theta chunks");
    if (is_fp64(c)) {
        if ((rc = upload_reals<double>(c, w.data(), c->d_thw, Nc))) return rc;
    } else {
        if ((rc = upload_reals<float>(c, w.data(), c->d_thw, Nc))) return rc;
    }
    c->nthchunk = (int)chunks.size();
    c->have_theta = true;
    return SHD_OK;
}

int shd_set_fields(shd_ctx *c, const double *alpha0, const double *ne, const double *u, const double *emis0,
                   const double *theta_e)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (!c->have_grid || !c->have_groups) return fail(SHD_ERR_STATE, "grid and groups must be set first");
    if (!alpha0 || !ne || !u || !emis0) return fail(SHD_ERR_ARG, "null field");
    if ((rc = ensure_buffers(c))) return rc;
    const size_t nCG = (size_t)c->Nc * c->G, Nc = (size_t)c->Nc;
    // the four fields as given (FP64) into a staging area, checked and
    // reduced there before any field array changes
    const size_t nf = 2 * nCG + 4 * Nc;
    if (c->fstage_n != nf || !c->d_fstage || !c->d_fcheck) {
        c->fstage_n = 0;
        if ((rc = dalloc(c, &c->d_fstage, nf * sizeof(double), "field staging"))) return rc;
        if ((rc = dalloc(c, &c->d_fcheck, sizeof(FieldCheck), "field check"))) return rc;
        c->fstage_n = nf;
    }
    double *sa = (double *)c->d_fstage, *se = sa + nCG, *sn = se + nCG, *su = sn + Nc;
    c->fstage_u_current = false;  // until these fields are accepted
    CK(cudaMemcpyAsync(sa, alpha0, nCG * sizeof(double), cudaMemcpyHostToDevice, c->stream), "H2D alpha0");
    CK(cudaMemcpyAsync(se, emis0, nCG * sizeof(double), cudaMemcpyHostToDevice, c->stream), "H2D emis0");
    CK(cudaMemcpyAsync(sn, ne, Nc * sizeof(double), cudaMemcpyHostToDevice, c->stream), "H2D ne");
    CK(cudaMemcpyAsync(su, u, 3 * Nc * sizeof(double), cudaMemcpyHostToDevice, c->stream), "H2D u");
    FieldCheck fc;
    const unsigned char *pm = c->have_fields ? c->d_mflag : nullptr;
    if (is_fp64(c)) CK(check_fields<double>(c, sa, sn, su, se, pm, c->have_fields ? (const double *)c->d_u : nullptr, fc), "field check");
    else CK(check_fields<float>(c, sa, sn, su, se, pm, c->have_fields ? (const float *)c->d_u : nullptr, fc), "field check");
    if (fc.bad & 1u) return fail(SHD_ERR_NAN, "alpha0 must be finite and >= 0");
    if (fc.bad & 2u) return fail(SHD_ERR_NAN, "ne must be finite and >= 0");
    if (fc.bad & 4u) return fail(SHD_ERR_NAN, "u must be finite");
    if (fc.bad & 8u) return fail(SHD_ERR_NAN, "emis0 must be finite and >= 0");
    double bits2d[3];
    std::memcpy(&bits2d[0], &fc.max_alpha, sizeof(double));
    std::memcpy(&bits2d[1], &fc.max_ne, sizeof(double));
    std::memcpy(&bits2d[2], &fc.max_uu, sizeof(double));
    c->h_alpha_max = bits2d[0];
    c->h_ne_max = bits2d[1];
    c->h_gamma_max = std::sqrt(1.0 + bits2d[2]);
    if (is_fp64(c)) {
        CK(launch_convert<double>(sa, (double *)c->d_alpha0, (long long)nCG, c->stream), "convert");
        CK(launch_convert<double>(se, (double *)c->d_emis0, (long long)nCG, c->stream), "convert");
        CK(launch_convert<double>(sn, (double *)c->d_ne, (long long)Nc, c->stream), "convert");
        CK(launch_convert<double>(su, (double *)c->d_u, (long long)(3 * Nc), c->stream), "convert");
    } else {
        CK(launch_convert<float>(sa, (float *)c->d_alpha0, (long long)nCG, c->stream), "convert");
        CK(launch_convert<float>(se, (float *)c->d_emis0, (long long)nCG, c->stream), "convert");
        CK(launch_convert<float>(sn, (float *)c->d_ne, (long long)Nc, c->stream), "convert");
        CK(launch_convert<float>(su, (float *)c->d_u, (long long)(3 * Nc), c->stream), "convert");
    }
    // the remap tables follow the flow in working precision: rebuilt before
    // the next step when it changed
    if (!c->have_fields || fc.u_changed) c->rtab_valid = false;
    // the node tables (and with them the captured step) change only when the
    // set of moving nodes does; new field values are read in place
    if (!c->have_fields || fc.moving_changed) {
        drop_graphs(c);
        c->rtab_valid = false;
        if ((rc = build_tiles(c, u))) return rc;
    }
    c->have_fields = true;
    c->fstage_u_current = true;
    if (theta_e) {
        if ((rc = set_theta(c, theta_e))) return rc;
    } else if (c->have_theta) {
        drop_graphs(c);
        c->have_theta = false;
        c->h_theta.clear();
        c->nthchunk = 0;
    }
    if (c->have_scat) {
        c->chi_rest_state = std::max(c->chi_rest_state, 1);  // chi0 may change: k_chi0_layout says
        if (is_fp64(c)) CK(launch_chi0<double>(c, c->stream), "chi0");
        else CK(launch_chi0<float>(c, c->stream), "chi0");
    }
    return SHD_OK;
}

int shd_set_scattering(shd_ctx *c, int kind, const double *K, const double *sigma_out)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    drop_graphs(c);  // the captured step holds the old parameters
    if (!c->have_angles || !c->have_groups) return fail(SHD_ERR_STATE, "angles and groups must be set first");
    if ((rc = ensure_buffers(c))) return rc;
    int G = c->G, L = c->L;
    size_t nK = (size_t)(L + 1) * G * G;
    std::vector<double> hK(nK, 0.0), hs(G, 1.0);
    if (kind == SHD_SCAT_ISO || kind == SHD_SCAT_THOMSON) {
        for (int g = 0; g < G; ++g) {
            hK[(size_t)g * G + g] = 1.0;
            if (kind == SHD_SCAT_THOMSON && L >= 2) hK[((size_t)2 * G + g) * G + g] = 0.1;
        }
    } else if (kind == SHD_SCAT_TABLE) {
        if (!K || !sigma_out) return fail(SHD_ERR_ARG, "table kind needs K and sigma_out");
        if (!finite_all(K, nK, false) || !finite_all(sigma_out, G, true))
            return fail(SHD_ERR_NAN, "scattering table must be finite (sigma_out >= 0)");
        hK.assign(K, K + nK);
        hs.assign(sigma_out, sigma_out + G);
    } else if (kind != SHD_SCAT_KN && kind != SHD_SCAT_KN_THERMAL) {
        return fail(SHD_ERR_ARG, "unknown scattering kind %d", kind);
    }
    if (kind == SHD_SCAT_KN_THERMAL && L > 15) return fail(SHD_ERR_ARG, "thermal Compton kernel needs L <= 15");
    if ((rc = dalloc(c, &c->d_K, nK * c->esize, "K"))) return rc;
    if ((rc = dalloc(c, &c->d_sigma_out, (size_t)G * c->esize, "sigma_out"))) return rc;
    if (kind == SHD_SCAT_KN_THERMAL) {
        // every temperature's table built on the device in FP64, then kept
        // in the working precision; K and sigma_out hold the coldest one
        std::vector<double> q, x, w;
        for (int n : {24, 16, 48, 16}) {  // electron speed, electron direction, scattering cosine, energy
            gauss_legendre(n, x, w);
            q.insert(q.end(), x.begin(), x.end());
            q.insert(q.end(), w.begin(), w.end());
        }
        const size_t nT = (size_t)kThermalN * nK;
        double *dK = nullptr, *ds = nullptr, *dq = nullptr;
        CK(cudaMalloc(&dK, sizeof(double) * nT), "thermal scratch");
        CK(cudaMalloc(&ds, sizeof(double) * kThermalN * G), "thermal scratch");
        CK(cudaMalloc(&dq, sizeof(double) * q.size()), "thermal scratch");
        CK(cudaMemcpy(dq, q.data(), sizeof(double) * q.size(), cudaMemcpyHostToDevice), "copy");
        CK(launch_kn_thermal_tables(G, c->d_edges, L, dq, dK, ds, c->stream), "thermal tables");
        if ((rc = dalloc(c, &c->d_thK, nT * c->esize, "thermal kernels"))) return rc;
        if ((rc = dalloc(c, &c->d_thso, (size_t)kThermalN * G * c->esize, "thermal cross-sections"))) return rc;
        if (is_fp64(c)) {
            CK(cudaMemcpyAsync(c->d_thK, dK, sizeof(double) * nT, cudaMemcpyDeviceToDevice, c->stream), "copy");
            CK(cudaMemcpyAsync(c->d_thso, ds, sizeof(double) * kThermalN * G, cudaMemcpyDeviceToDevice, c->stream), "copy");
            CK(cudaMemcpyAsync(c->d_K, dK, sizeof(double) * nK, cudaMemcpyDeviceToDevice, c->stream), "copy");
            CK(cudaMemcpyAsync(c->d_sigma_out, ds, sizeof(double) * G, cudaMemcpyDeviceToDevice, c->stream), "copy");
        } else {
            CK(launch_convert<float>(dK, (float *)c->d_thK, (long long)nT, c->stream), "convert");
            CK(launch_convert<float>(ds, (float *)c->d_thso, (long long)kThermalN * G, c->stream), "convert");
            CK(launch_convert<float>(dK, (float *)c->d_K, (long long)nK, c->stream), "convert");
            CK(launch_convert<float>(ds, (float *)c->d_sigma_out, G, c->stream), "convert");
        }
        CK(cudaStreamSynchronize(c->stream), "sync");
        std::vector<double> hso((size_t)kThermalN * G);
        CK(cudaMemcpy(hso.data(), ds, sizeof(double) * hso.size(), cudaMemcpyDeviceToHost), "sigma_out");
        c->h_sigma_max = 0.0;
        for (double v : hso) c->h_sigma_max = std::max(c->h_sigma_max, v);
        cudaFree(dK); cudaFree(ds); cudaFree(dq);
    } else if (kind == SHD_SCAT_KN) {
        // built on the device in FP64, then converted to the working precision
        const int nq = 32;
        std::vector<double> gx, gw;
        gauss_legendre(nq, gx, gw);
        double *dK = nullptr, *ds = nullptr, *dgx = nullptr, *dgw = nullptr;
        CK(cudaMalloc(&dK, sizeof(double) * nK), "KN scratch");
        CK(cudaMalloc(&ds, sizeof(double) * G), "KN scratch");
        CK(cudaMalloc(&dgx, sizeof(double) * nq), "KN scratch");
        CK(cudaMalloc(&dgw, sizeof(double) * nq), "KN scratch");
        CK(cudaMemcpy(dgx, gx.data(), sizeof(double) * nq, cudaMemcpyHostToDevice), "copy");
        CK(cudaMemcpy(dgw, gw.data(), sizeof(double) * nq, cudaMemcpyHostToDevice), "copy");
        CK(launch_kn_table(G, c->d_edges, L, dK, ds, dgx, dgw, nq, c->stream), "kn_table");
        if (is_fp64(c)) {
            CK(cudaMemcpyAsync(c->d_K, dK, sizeof(double) * nK, cudaMemcpyDeviceToDevice, c->stream), "copy");
            CK(cudaMemcpyAsync(c->d_sigma_out, ds, sizeof(double) * G, cudaMemcpyDeviceToDevice, c->stream), "copy");
        } else {
            CK(launch_convert<float>(dK, (float *)c->d_K, (long long)nK, c->stream), "convert");
            CK(launch_convert<float>(ds, (float *)c->d_sigma_out, G, c->stream), "convert");
        }
        CK(cudaStreamSynchronize(c->stream), "sync");
        std::vector<double> hso(G);
        CK(cudaMemcpy(hso.data(), ds, sizeof(double) * G, cudaMemcpyDeviceToHost), "sigma_out");
        c->h_sigma_max = 0.0;
        for (double v : hso) c->h_sigma_max = std::max(c->h_sigma_max, v);
        cudaFree(dK); cudaFree(ds); cudaFree(dgx); cudaFree(dgw);
    } else {
        c->h_sigma_max = 0.0;
        for (double v : hs) c->h_sigma_max = std::max(c->h_sigma_max, v);
        if (is_fp64(c)) {
            if ((rc = upload_reals<double>(c, hK.data(), c->d_K, nK))) return rc;
            if ((rc = upload_reals<double>(c, hs.data(), c->d_sigma_out, G))) return rc;
        } else {
            if ((rc = upload_reals<float>(c, hK.data(), c->d_K, nK))) return rc;
            if ((rc = upload_reals<float>(c, hs.data(), c->d_sigma_out, G))) return rc;
        }
    }
    c->scat_kind = kind;
    // the source stage's one-product form needs every K_l diagonal
    c->k_diagonal = kind != SHD_SCAT_KN && kind != SHD_SCAT_KN_THERMAL;
    if (kind == SHD_SCAT_TABLE)
        for (size_t i = 0; i < nK && c->k_diagonal; ++i) {
            const size_t r = i % ((size_t)G * G);
            if (r / G != r % G && hK[i] != 0.0) c->k_diagonal = false;
        }
    c->have_scat = true;
    // the tensor-core source's BF16 operands of a group-mixing kernel
    dfree(c->d_tcK);
    c->source_choice = 0;
    if (c->precision == SHD_MIXED && !c->k_diagonal && kind != SHD_SCAT_KN_THERMAL) {
        if ((rc = dalloc(c, &c->d_tcK, source_tc_operand_bytes(c), "source operands"))) return rc;
        CK(launch_source_tc_operands(c, c->stream), "source operands");
    }
    if (c->have_fields) {
        c->chi_rest_state = std::max(c->chi_rest_state, 1);  // chi0 may change: k_chi0_layout says
        if (is_fp64(c)) CK(launch_chi0<double>(c, c->stream), "chi0");
        else CK(launch_chi0<float>(c, c->stream), "chi0");
    }
    return SHD_OK;
}

int shd_get_scattering(shd_ctx *c, double *K, double *sigma_out)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (!c->have_scat) return fail(SHD_ERR_STATE, "scattering not set");
    size_t nK = (size_t)(c->L + 1) * c->G * c->G;
    if (is_fp64(c)) {
        if (K && (rc = download_reals<double>(c, c->d_K, K, nK))) return rc;
        if (sigma_out && (rc = download_reals<double>(c, c->d_sigma_out, sigma_out, c->G))) return rc;
    } else {
        if (K && (rc = download_reals<float>(c, c->d_K, K, nK))) return rc;
        if (sigma_out && (rc = download_reals<float>(c, c->d_sigma_out, sigma_out, c->G))) return rc;
    }
    return SHD_OK;
}

int shd_set_boundary(shd_ctx *c, int mode, const double *data)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    drop_graphs(c);  // the captured step holds the old parameters
    if (mode == SHD_BC_VACUUM) {
        dfree(c->d_bc);
        c->bc_mode = mode;
        return SHD_OK;
    }
    if (!sized(c)) return fail(SHD_ERR_STATE, "grid, angles and groups must be set first");
    if (!data) return fail(SHD_ERR_ARG, "boundary data is NULL");
    if ((rc = ensure_buffers(c))) return rc;
    if (mode == SHD_BC_ISO) {
        if (!finite_all(data, c->G, true)) return fail(SHD_ERR_NAN, "boundary intensity must be finite and >= 0");
        if ((rc = dalloc(c, &c->d_bc, (size_t)c->G * c->esize, "bc"))) return rc;
        rc = is_fp64(c) ? upload_reals<double>(c, data, c->d_bc, c->G) : upload_reals<float>(c, data, c->d_bc, c->G);
        if (rc) return rc;
    } else if (mode == SHD_BC_FULL) {
        size_t n = (size_t)c->Nc * c->G * c->N;
        if (!finite_all(data, n, false)) return fail(SHD_ERR_NAN, "boundary intensity must be finite");
        if ((rc = dalloc(c, &c->d_bc, n * c->esize, "bc"))) return rc;
        rc = is_fp64(c) ? set_state_impl<double>(c, data, true, c->stream, (double *)c->d_bc)
                        : set_state_impl<float>(c, data, true, c->stream, (float *)c->d_bc);
        if (rc) return rc;
    } else {
        return fail(SHD_ERR_ARG, "unknown boundary mode %d", mode);
    }
    c->bc_mode = mode;
    CK(cudaStreamSynchronize(c->stream), "sync");
    return SHD_OK;
}

int shd_set_time(shd_ctx *c, double kappa)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    drop_graphs(c);  // the captured step holds the old parameters
    if (!std::isfinite(kappa) || kappa < 0) return fail(SHD_ERR_ARG, "kappa must be finite and >= 0");
    c->kappa = kappa;
    return SHD_OK;
}

int shd_set_state(shd_ctx *c, const double *I)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (!I) return fail(SHD_ERR_ARG, "I is NULL");
    if ((rc = ensure_buffers(c))) return rc;
    rc = is_fp64(c) ? set_state_impl<double>(c, I, true, c->stream, (double *)c->d_I)
                    : set_state_impl<float>(c, I, true, c->stream, (float *)c->d_I);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream), "sync");
    c->have_state = true;
    c->sprev_valid = false;
    return SHD_OK;
}

int shd_set_state_dev(shd_ctx *c, const double *dev_I, void *stream)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (!dev_I) return fail(SHD_ERR_ARG, "dev_I is NULL");
    if ((rc = ensure_buffers(c))) return rc;
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    if ((rc = stream_after(st, c->stream))) return rc;
    rc = is_fp64(c) ? set_state_impl<double>(c, dev_I, false, st, (double *)c->d_I)
                    : set_state_impl<float>(c, dev_I, false, st, (float *)c->d_I);
    if (rc) return rc;
    if ((rc = stream_after(c->stream, st))) return rc;
    c->have_state = true;
    c->sprev_valid = false;
    return SHD_OK;
}

int shd_zero_state(shd_ctx *c)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if ((rc = ensure_buffers(c))) return rc;
    CK(cudaMemsetAsync(c->d_I, 0, (size_t)c->Nc * c->G * c->N * c->esize, c->stream), "memset");
    c->have_state = true;
    c->sprev_valid = false;
    return SHD_OK;
}

int shd_get_state(shd_ctx *c, double *I)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (!I) return fail(SHD_ERR_ARG, "I is NULL");
    if (!c->have_state) return fail(SHD_ERR_STATE, "state not set");
    return is_fp64(c) ? get_state_impl<double>(c, (const double *)c->d_I, I, true, c->stream)
                      : get_state_impl<float>(c, (const float *)c->d_I, I, true, c->stream);
}

int shd_get_state_dev(shd_ctx *c, double *dev_I, void *stream)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (!dev_I) return fail(SHD_ERR_ARG, "dev_I is NULL");
    if (!c->have_state) return fail(SHD_ERR_STATE, "state not set");
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    if ((rc = stream_after(st, c->stream))) return rc;
    return is_fp64(c) ? get_state_impl<double>(c, (const double *)c->d_I, dev_I, false, st)
                      : get_state_impl<float>(c, (const float *)c->d_I, dev_I, false, st);
}

int shd_step(shd_ctx *c, int nsteps, void *stream)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (nsteps < 0) return fail(SHD_ERR_ARG, "nsteps < 0");
    if ((rc = ready_for_step(c))) return rc;
    if (!c->have_state) return fail(SHD_ERR_STATE, "state not set");
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    // order against the library's own stream (uploads, reads) both ways
    if ((rc = stream_after(st, c->stream))) return rc;
    rc = is_fp64(c) ? run_steps<double>(c, nsteps, st, true) : run_steps<float>(c, nsteps, st, true);
    if (rc) return rc;
    return stream_after(c->stream, st);
}

int shd_solve_static(shd_ctx *c, double rel_tol, int max_iter, int *iters_out, double *resid_out)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (!(rel_tol > 0) || max_iter < 1) return fail(SHD_ERR_ARG, "need rel_tol > 0 and max_iter >= 1");
    if ((rc = ready_for_step(c))) return rc;
    if (!c->have_state && (rc = shd_zero_state(c))) return rc;
    // Ng acceleration: the last three source iterates and the scratch of
    // the inner products
    const size_t nS = (size_t)c->Nc * c->G * c->NLM;
    const int ng_blocks = 4 * 152;
    if (c->ng_period >= 4) {
        for (int i = 0; i < 3; ++i)
            if (!c->d_ng[i] && (rc = dalloc(c, &c->d_ng[i], nS * c->esize, "Ng iterates"))) return rc;
        if (!c->d_ngpart && (rc = dalloc(c, (void **)&c->d_ngpart, sizeof(double) * (5 * ng_blocks + 5), "Ng sums")))
            return rc;
    }
    double kap = c->kappa;
    c->kappa = 0.0;
    c->sprev_valid = false;
    int it = 0, last_ng = 0;
    double sums[3] = {0, 0, 0};
    // Ng (Sec. 2; Ng 1974) on iterate it = S^it, just formed by the source
    // stage: at it >= 4 with it - last_ng >= period, x* = (1 - a - b) S^it +
    // a S^(it-1) + b S^(it-2), (a, b) minimising |Q3 - a Q1 - b Q2| (FP64
    // inner products; skipped when that 2 x 2 system is singular); then
    // S^it (or x*) is kept as the newest of the three stored iterates
    std::function<int()> ng_step = [&]() -> int {
        const int n = it + 1;  // the iterate being formed
        auto slot = [&](int j) { return c->d_ng[((j % 3) + 3) % 3]; };
        if (n >= 4 && n - last_ng >= c->ng_period) {
            double d[5];
            cudaError_t e = is_fp64(c)
                ? launch_ng_dots<double>((const double *)c->d_Sp, (const double *)slot(n - 1),
                                         (const double *)slot(n - 2), (const double *)slot(n - 3), (long long)nS,
                                         c->d_ngpart, ng_blocks, c->d_ngpart + 5 * ng_blocks, c->stream)
                : launch_ng_dots<float>((const float *)c->d_Sp, (const float *)slot(n - 1),
                                        (const float *)slot(n - 2), (const float *)slot(n - 3), (long long)nS,
                                        c->d_ngpart, ng_blocks, c->d_ngpart + 5 * ng_blocks, c->stream);
            if (e == cudaSuccess)
                e = cudaMemcpyAsync(d, c->d_ngpart + 5 * ng_blocks, sizeof(d), cudaMemcpyDeviceToHost, c->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
            if (e != cudaSuccess) return cuda_fail(e, "Ng inner products");
            const double det = d[0] * d[2] - d[1] * d[1];
            if (std::isfinite(det) && det > 1e-14 * d[0] * d[2]) {
                const double a = (d[3] * d[2] - d[4] * d[1]) / det;
                const double b = (d[4] * d[0] - d[3] * d[1]) / det;
                e = is_fp64(c) ? launch_ng_combine<double>((double *)c->d_Sp, (const double *)slot(n - 1),
                                                           (const double *)slot(n - 2), (long long)nS, a, b, c->stream)
                               : launch_ng_combine<float>((float *)c->d_Sp, (const float *)slot(n - 1),
                                                          (const float *)slot(n - 2), (long long)nS, a, b, c->stream);
                if (e != cudaSuccess) return cuda_fail(e, "Ng extrapolation");
                last_ng = n;
            }
        }
        CK(cudaMemcpyAsync(slot(n), c->d_Sp, nS * c->esize, cudaMemcpyDeviceToDevice, c->stream), "Ng iterate");
        return SHD_OK;
    };
    const std::function<int()> *hook = c->ng_period >= 4 ? &ng_step : nullptr;
    const int scheme = c->time_scheme;
    c->time_scheme = SHD_TIME_EULER;  // the static iteration has no time term to sub-step
    while (it < max_iter) {
        rc = is_fp64(c) ? run_steps<double>(c, 1, c->stream, false, hook)
                        : run_steps<float>(c, 1, c->stream, false, hook);
        if (rc) break;
        ++it;
        cudaError_t e = cudaMemcpyAsync(sums, c->d_sums, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream);
        if (e == cudaSuccess) e = cudaStreamSynchronize(c->stream);
        if (e != cudaSuccess) { rc = cuda_fail(e, "residual read"); break; }
        if (it > 1 && sums[2] <= rel_tol) break;
    }
    c->time_scheme = scheme;
    c->kappa = kap;
    if (iters_out) *iters_out = it;
    if (resid_out) *resid_out = sums[2];
    if (rc) return rc;
    if (!(sums[2] <= rel_tol)) return fail(SHD_ERR_TIMEOUT, "not converged after %d iterations (resid %g)", it, sums[2]);
    return SHD_OK;
}

int shd_get_moments(shd_ctx *c, double *J, double *H, double *K, double *Ish)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if ((rc = ready_for_step(c))) return rc;
    if (!c->have_state) return fail(SHD_ERR_STATE, "state not set");
    size_t nCG = (size_t)c->Nc * c->G;
    std::vector<double> mom(nCG * 10);
    if (is_fp64(c)) {
        CK(launch_project<double>(c, (const double *)c->d_I, (double *)c->d_Ip, (double *)c->d_mom, c->stream), "project");
        if ((rc = download_reals<double>(c, c->d_mom, mom.data(), nCG * 10))) return rc;
        if (Ish && (rc = download_reals<double>(c, c->d_Ip, Ish, nCG * c->NLM))) return rc;
    } else {
        CK(launch_project<float>(c, (const float *)c->d_I, (float *)c->d_Ip, (float *)c->d_mom, c->stream), "project");
        if ((rc = download_reals<float>(c, c->d_mom, mom.data(), nCG * 10))) return rc;
        if (Ish && (rc = download_reals<float>(c, c->d_Ip, Ish, nCG * c->NLM))) return rc;
    }
    if ((rc = check_device_flags(c))) return rc;
    for (size_t i = 0; i < nCG; ++i) {
        if (J) J[i] = mom[i * 10];
        if (H) for (int q = 0; q < 3; ++q) H[i * 3 + q] = mom[i * 10 + 1 + q];
        if (K) for (int q = 0; q < 6; ++q) K[i * 6 + q] = mom[i * 10 + 4 + q];
    }
    return SHD_OK;
}

}  // extern "C"

namespace {
// working-precision moments into the caller's FP64 array (an exact widening)
template <class T>
__global__ void k_widen(const T *__restrict__ src, double *__restrict__ dst, long long n)
{
    for (long long i = (long long)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        dst[i] = (double)src[i];
}
}  // namespace

extern "C" {

int shd_get_moments_dev(shd_ctx *c, double *dev_mom, void *stream)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (!dev_mom) return fail(SHD_ERR_ARG, "dev_mom is NULL");
    if ((rc = ready_for_step(c))) return rc;
    if (!c->have_state) return fail(SHD_ERR_STATE, "state not set");
    cudaStream_t st = stream ? (cudaStream_t)stream : c->stream;
    if ((rc = stream_after(st, c->stream))) return rc;
    const long long n = (long long)c->Nc * c->G * 10;
    const unsigned blocks = (unsigned)std::min<long long>((n + 255) / 256, 4LL * 152);
    if (is_fp64(c)) {
        CK(launch_project<double>(c, (const double *)c->d_I, (double *)c->d_Ip, (double *)c->d_mom, st), "project");
        CK(cudaMemcpyAsync(dev_mom, c->d_mom, n * sizeof(double), cudaMemcpyDeviceToDevice, st), "moments");
    } else {
        CK(launch_project<float>(c, (const float *)c->d_I, (float *)c->d_Ip, (float *)c->d_mom, st), "project");
        k_widen<float><<<blocks, 256, 0, st>>>((const float *)c->d_mom, dev_mom, n);
        note_launch();
        CK(cudaGetLastError(), "moments");
    }
    return stream_after(c->stream, st);
}

int shd_get_sums(shd_ctx *c, double *energy, double *photons, double *resid)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if ((rc = check_device_flags(c))) return rc;
    double s[3];
    CK(cudaMemcpyAsync(s, c->d_sums, sizeof(double) * 3, cudaMemcpyDeviceToHost, c->stream), "D2H sums");
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (energy) *energy = s[0];
    if (photons) *photons = s[1];
    if (resid) *resid = s[2];
    return SHD_OK;
}

int shd_set_ng(shd_ctx *c, int period)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (period != 0 && period < 4) return fail(SHD_ERR_ARG, "Ng period must be 0 (off) or >= 4");
    c->ng_period = period;
    return SHD_OK;
}

int shd_set_time_scheme(shd_ctx *c, int scheme)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (scheme != SHD_TIME_EULER && scheme != SHD_TIME_RK4) return fail(SHD_ERR_ARG, "unknown time scheme %d", scheme);
    if (scheme != c->time_scheme) drop_graphs(c);
    c->time_scheme = scheme;
    if (scheme == SHD_TIME_EULER) {
        for (int i = 0; i < 3; ++i) dfree(c->d_rk[i]);
        return SHD_OK;
    }
    if (sized(c)) return ensure_rk_buffers(c);
    return SHD_OK;
}

int shd_get_thermal_tables(shd_ctx *c, double *K_th, double *sigma_out_th)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (c->scat_kind != SHD_SCAT_KN_THERMAL || !c->d_thK) return fail(SHD_ERR_STATE, "no thermal Compton kernel set");
    const size_t nT = (size_t)kThermalN * (c->L + 1) * c->G * c->G, nS = (size_t)kThermalN * c->G;
    if (K_th) {
        if (is_fp64(c)) { if ((rc = download_reals<double>(c, c->d_thK, K_th, nT))) return rc; }
        else if ((rc = download_reals<float>(c, c->d_thK, K_th, nT))) return rc;
    }
    if (sigma_out_th) {
        if (is_fp64(c)) { if ((rc = download_reals<double>(c, c->d_thso, sigma_out_th, nS))) return rc; }
        else if ((rc = download_reals<float>(c, c->d_thso, sigma_out_th, nS))) return rc;
    }
    return SHD_OK;
}

int shd_set_integrator(shd_ctx *c, int integrator)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (integrator != SHD_SC_LINEAR && integrator != SHD_SC_BEZIER)
        return fail(SHD_ERR_ARG, "unknown integrator %d", integrator);
    if (integrator != c->integrator) drop_graphs(c);
    c->integrator = integrator;
    return SHD_OK;
}

int shd_set_sweep_schedule(shd_ctx *c, int C, int NT)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (C == 0) {
        c->sweep_force_C = c->sweep_force_NT = 0;
        c->sweep_C = c->sweep_NT = 0;  // choose again on the next sweep
        drop_graphs(c);
        return SHD_OK;
    }
    if (!sized(c)) return fail(SHD_ERR_STATE, "grid, angles and groups must be set");
    if (!sweep_schedule_valid(c, C, NT))
        return fail(SHD_ERR_ARG, "sweep schedule C=%d NT=%d does not fit this problem (or it has no FP32 plane sweep)",
                    C, NT);
    c->sweep_force_C = C;
    c->sweep_force_NT = NT;
    drop_graphs(c);
    return SHD_OK;
}

int shd_get_sweep_schedule(shd_ctx *c, int *C, int *NT, int *ncand, float *cand)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (C) *C = c->sweep_force_C ? c->sweep_force_C : c->sweep_C;
    if (NT) *NT = c->sweep_force_C ? c->sweep_force_NT : c->sweep_NT;
    if (ncand) *ncand = c->sweep_ntune;
    if (cand)
        for (int i = 0; i < c->sweep_ntune; ++i)
            for (int q = 0; q < 3; ++q) cand[3 * i + q] = c->sweep_tune[i][q];
    return SHD_OK;
}

int shd_set_source_path(shd_ctx *c, int path)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (path < 0 || path > 2) return fail(SHD_ERR_ARG, "source path must be 0 (timed), 1 (CUDA cores) or 2 (tensor cores)");
    if (path == 2 && !source_tc_usable(c))
        return fail(SHD_ERR_ARG, "no tensor-core source for this problem (MIXED with a group-mixing kernel, "
                                 "operands within shared memory)");
    c->source_choice = path;
    drop_graphs(c);
    return SHD_OK;
}

int shd_get_source_path(shd_ctx *c, int *path, float *ms_cuda_cores, float *ms_tensor_cores)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (path) *path = source_tc_usable(c) ? c->source_choice : 1;
    if (ms_cuda_cores) *ms_cuda_cores = c->source_ms[0];
    if (ms_tensor_cores) *ms_tensor_cores = c->source_ms[1];
    return SHD_OK;
}

int shd_get_transform_path(shd_ctx *c, int *path)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (!sized(c)) return fail(SHD_ERR_STATE, "grid, angles and groups must be set");
    int p = 0;
    if (c->precision == SHD_MIXED) {
        if (seg_usable(c)) p = seg_manual(c) ? 3 : 2;
        else if (tc_usable(c)) p = 1;
    }
    if (path) *path = p;
    return SHD_OK;
}

int shd_check_bounded_wait(shd_ctx *c, long long polls)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if (polls < 1 || polls > (1LL << 22)) return fail(SHD_ERR_ARG, "polls must be in [1, 2^22]");
    if ((rc = check_device_flags(c))) return rc;  // report (and clear) an earlier give-up first
    CK(launch_wait_selftest(polls, c->d_tc_err, c->stream), "wait self-check");
    return check_device_flags(c);
}

// ---- single stages --------------------------------------------------------

int shd_stage_project(shd_ctx *c, const double *I, double *Ish, double *J, double *H, double *K)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if ((rc = ready_for_step(c))) return rc;
    if ((rc = ensure_remap_tables(c, nullptr))) return rc;  // the remaps as a step runs them
    if (!I) return fail(SHD_ERR_ARG, "I is NULL");
    if ((rc = shd_set_state(c, I))) return rc;
    return shd_get_moments(c, J, H, K, Ish);
}

int shd_stage_source(shd_ctx *c, const double *Ish, double *Ssh)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if ((rc = ready_for_step(c))) return rc;
    if (!Ish || !Ssh) return fail(SHD_ERR_ARG, "null array");
    size_t n = (size_t)c->Nc * c->G * c->NLM;
    if (is_fp64(c)) {
        if ((rc = upload_reals<double>(c, Ish, c->d_Ip, n))) return rc;
        CK(launch_source<double>(c, (const double *)c->d_Ip, (double *)c->d_Sp, c->stream), "source");
        return download_reals<double>(c, c->d_Sp, Ssh, n);
    }
    if ((rc = upload_reals<float>(c, Ish, c->d_Ip, n))) return rc;
    CK(launch_source<float>(c, (const float *)c->d_Ip, (float *)c->d_Sp, c->stream), "source");
    return download_reals<float>(c, c->d_Sp, Ssh, n);
}

int shd_stage_sh2lab(shd_ctx *c, const double *Ssh, double *eta_lab, double *chi_lab)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if ((rc = ready_for_step(c))) return rc;
    if ((rc = ensure_remap_tables(c, nullptr))) return rc;  // the remaps as a step runs them
    if (!Ssh || !eta_lab || !chi_lab) return fail(SHD_ERR_ARG, "null array");
    size_t n = (size_t)c->Nc * c->G * c->NLM;
    if (is_fp64(c)) {
        if ((rc = upload_reals<double>(c, Ssh, c->d_Sp, n))) return rc;
        CK(launch_sh2lab<double>(c, (const double *)c->d_Sp, (double *)c->d_eta, (double *)c->d_chi, c->stream), "sh2lab");
        if ((rc = get_state_impl<double>(c, (const double *)c->d_eta, eta_lab, true, c->stream))) return rc;
        return get_state_impl<double>(c, (const double *)c->d_chi, chi_lab, true, c->stream);
    }
    if ((rc = upload_reals<float>(c, Ssh, c->d_Sp, n))) return rc;
    CK(launch_sh2lab<float>(c, (const float *)c->d_Sp, (float *)c->d_eta, (float *)c->d_chi, c->stream), "sh2lab");
    if ((rc = get_state_impl<float>(c, (const float *)c->d_eta, eta_lab, true, c->stream))) return rc;
    return get_state_impl<float>(c, (const float *)c->d_chi, chi_lab, true, c->stream);
}

int shd_stage_sweep(shd_ctx *c, const double *I_old, const double *eta_lab, const double *chi_lab, double *I_new)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    if ((rc = ready_for_step(c))) return rc;
    if (!I_old || !eta_lab || !chi_lab || !I_new) return fail(SHD_ERR_ARG, "null array");
    c->chi_rest_state = 2;  // chi_lab becomes the caller's: the next step fills chi0 at rest again
    if (is_fp64(c)) {
        if ((rc = set_state_impl<double>(c, eta_lab, true, c->stream, (double *)c->d_eta))) return rc;
        if ((rc = set_state_impl<double>(c, chi_lab, true, c->stream, (double *)c->d_chi))) return rc;
        if ((rc = set_state_impl<double>(c, I_old, true, c->stream, (double *)c->d_I))) return rc;
        CK(launch_sweep<double>(c, (double *)c->d_I, (const double *)c->d_eta, (const double *)c->d_chi, c->stream), "sweep");
    } else {
        if ((rc = set_state_impl<float>(c, eta_lab, true, c->stream, (float *)c->d_eta))) return rc;
        if ((rc = set_state_impl<float>(c, chi_lab, true, c->stream, (float *)c->d_chi))) return rc;
        if ((rc = set_state_impl<float>(c, I_old, true, c->stream, (float *)c->d_I))) return rc;
        CK(launch_sweep<float>(c, (float *)c->d_I, (const float *)c->d_eta, (const float *)c->d_chi, c->stream), "sweep");
    }
    c->have_state = true;
    return shd_get_state(c, I_new);
}

int shd_get_sizes(shd_ctx *c, long long *n_nodes, int *n_ord, int *n_groups, int *n_lm)
{
    if (!c) return fail(SHD_ERR_ARG, "null context");
    if (n_nodes) *n_nodes = c->Nc;
    if (n_ord) *n_ord = c->N;
    if (n_groups) *n_groups = c->G;
    if (n_lm) *n_lm = c->NLM;
    return SHD_OK;
}

long long shd_device_bytes(shd_ctx *c) { return c ? c->bytes : 0; }

int shd_set_timing(shd_ctx *c, int on)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    CK(cudaStreamSynchronize(c->stream), "sync");
    if (on && c->timing.pool.empty()) {
        c->timing.pool.assign((size_t)Timing::kCap * (Timing::kStages + 1), nullptr);
        for (cudaEvent_t &e : c->timing.pool) CK(cudaEventCreate(&e), "cudaEventCreate");
    }
    c->timing.on = on != 0;
    c->timing.count = 0;
    return SHD_OK;
}

int shd_get_timing(shd_ctx *c, double *stage_ms, long long *steps)
{
    int rc = ctx_check(c);
    if (rc) return rc;
    double ms[Timing::kStages] = {0, 0, 0, 0, 0};
    long long n = c->timing.count;
    if (n > 0) {
        CK(cudaEventSynchronize(c->timing.pool[(size_t)(n - 1) * (Timing::kStages + 1) + Timing::kStages]), "sync");
        for (long long s = 0; s < n; ++s) {
            cudaEvent_t *ev = &c->timing.pool[(size_t)s * (Timing::kStages + 1)];
            for (int q = 0; q < Timing::kStages; ++q) {
                float t = 0;
                CK(cudaEventElapsedTime(&t, ev[q], ev[q + 1]), "elapsed");
                ms[q] += t;
            }
        }
    }
    if (stage_ms)
        for (int q = 0; q < Timing::kStages; ++q) stage_ms[q] = ms[q];
    if (steps) *steps = n;
    return SHD_OK;
}

// ---------------------------------------------------------------------------
// batches of independent problems
// ---------------------------------------------------------------------------
}  // extern "C"

struct shd_batch {
    std::vector<shd_ctx *> probs;
    int device = 0;
    int sweep_mode = 0;  // 1: one plane-sweep launch per class of problems
    // cached graphs of one batch step: the key is each problem's graph
    // generation, slot (-1: that problem steps by direct launches) and
    // sweep class (0: the problem's graph holds its own sweep; otherwise the
    // slot is that of its sweep-less graph and the class's launch sweeps it)
    struct Key {
        unsigned long long gen;
        int slot, cls;
        bool operator==(const Key &o) const { return gen == o.gen && slot == o.slot && cls == o.cls; }
    };
    struct Entry {
        std::vector<Key> key;
        cudaGraphExec_t exec = nullptr;
        std::vector<void *> desc;    // device work lists of the batched sweeps
        unsigned long long extra = 0;  // kernels of those sweeps per launch
    };
    std::vector<Entry> cache;
};

namespace {
void batch_drop(shd_batch *b)
{
    bool lists = false;
    for (auto &e : b->cache) lists |= !e.desc.empty();
    if (lists) cudaDeviceSynchronize();  // a launched step may still read its work lists
    for (auto &e : b->cache) {
        if (e.exec) cudaGraphExecDestroy(e.exec);
        for (void *d : e.desc) cudaFree(d);
    }
    b->cache.clear();
}

// The batch graph of one step for key: each problem's step (or its
// sweep-less step) as a child graph, and per sweep class one persistent
// plane sweep over the work list of its problems' (ordinate, group) pairs,
// after their sweep-less steps.  The work list is ordered by falling node
// count, so that the static stride of the persistent CTAs meets the long
// items first.
int batch_build(shd_batch *b, const std::vector<shd_batch::Key> &key, shd_batch::Entry &ent)
{
    const int np = (int)b->probs.size();
    cudaGraph_t bg = nullptr;
    CK(cudaGraphCreate(&bg, 0), "batch graph");
    cudaError_t e = cudaSuccess;
    std::vector<cudaGraphNode_t> node(np, nullptr);
    for (int p = 0; p < np && e == cudaSuccess; ++p) {
        if (key[p].slot < 0) continue;
        shd_ctx *c = b->probs[p];
        cudaGraph_t child = key[p].cls ? c->graph_ns[key[p].slot] : c->graph[key[p].slot];
        e = cudaGraphAddChildGraphNode(&node[p], bg, nullptr, 0, child);
    }
    std::vector<int> classes;
    for (int p = 0; p < np; ++p)
        if (key[p].slot >= 0 && key[p].cls && std::find(classes.begin(), classes.end(), key[p].cls) == classes.end())
            classes.push_back(key[p].cls);
    cudaStream_t cs = nullptr;
    for (size_t q = 0; q < classes.size() && e == cudaSuccess; ++q) {
        const int cls = classes[q];
        std::vector<int> mem;
        for (int p = 0; p < np; ++p)
            if (key[p].slot >= 0 && key[p].cls == cls) mem.push_back(p);
        std::stable_sort(mem.begin(), mem.end(), [&](int x, int y) { return b->probs[x]->Nc > b->probs[y]->Nc; });
        std::vector<SweepBatchProb> h(mem.size());
        std::vector<cudaGraphNode_t> deps;
        long long items = 0;
        size_t smem = 0;
        for (size_t k = 0; k < mem.size(); ++k) {
            shd_ctx *c = b->probs[mem[k]];
            sweep_batch_fill(c, h[k], items);
            items += (long long)c->N * c->G;
            smem = std::max(smem, sweep_batch_smem(c));
            deps.push_back(node[mem[k]]);
        }
        void *d = nullptr;
        e = cudaMalloc(&d, h.size() * sizeof(SweepBatchProb));
        if (e != cudaSuccess) break;
        ent.desc.push_back(d);
        e = cudaMemcpy(d, h.data(), h.size() * sizeof(SweepBatchProb), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) break;
        if (!cs && (e = cudaStreamCreateWithFlags(&cs, cudaStreamNonBlocking)) != cudaSuccess) break;
        const unsigned long long n0 = shd_launch_count_now();
        e = cudaStreamBeginCapture(cs, cudaStreamCaptureModeThreadLocal);
        if (e != cudaSuccess) break;
        const cudaError_t el = launch_sweep_batch(cls, (const SweepBatchProb *)d, (int)h.size(), items, smem,
                                                  b->device, cs);
        cudaGraph_t sg = nullptr;
        e = cudaStreamEndCapture(cs, &sg);
        const unsigned long long n = shd_launch_count_now() - n0;
        forget_launches(n);
        ent.extra += n;
        if (e == cudaSuccess) e = el;
        if (e == cudaSuccess) {
            cudaGraphNode_t sn;
            e = cudaGraphAddChildGraphNode(&sn, bg, deps.data(), deps.size(), sg);
        }
        if (sg) cudaGraphDestroy(sg);
    }
    if (cs) cudaStreamDestroy(cs);
    if (e == cudaSuccess) e = cudaGraphInstantiate(&ent.exec, bg, 0);
    cudaGraphDestroy(bg);
    if (e != cudaSuccess) {
        for (void *d : ent.desc) cudaFree(d);
        ent.desc.clear();
        ent.exec = nullptr;
        return cuda_fail(e, "batch graph");
    }
    return SHD_OK;
}
}  // namespace

extern "C" {

int shd_batch_create(shd_batch **out, int nprob, shd_ctx *const *problems)
{
    if (!out) return fail(SHD_ERR_ARG, "out is NULL");
    *out = nullptr;
    if (nprob < 1 || !problems) return fail(SHD_ERR_ARG, "need at least one problem");
    for (int i = 0; i < nprob; ++i) {
        if (!problems[i]) return fail(SHD_ERR_ARG, "problem %d is NULL", i);
        if (problems[i]->device != problems[0]->device) return fail(SHD_ERR_ARG, "problems on different devices");
    }
    shd_batch *b = new (std::nothrow) shd_batch;
    if (!b) return fail(SHD_ERR_OOM, "batch");
    b->probs.assign(problems, problems + nprob);
    b->device = problems[0]->device;
    *out = b;
    return SHD_OK;
}

int shd_batch_step(shd_batch *b, int nsteps, void *stream)
{
    if (!b) return fail(SHD_ERR_ARG, "null batch");
    if (nsteps < 0) return fail(SHD_ERR_ARG, "nsteps < 0");
    CK(cudaSetDevice(b->device), "cudaSetDevice");
    const int np = (int)b->probs.size();
    for (int p = 0; p < np; ++p) {
        shd_ctx *c = b->probs[p];
        int rc = ready_for_step(c);
        if (!rc && !c->have_state) rc = fail(SHD_ERR_STATE, "state not set");
        if (rc) return fail(rc, "problem %d: %s", p, std::string(g_err).c_str());
    }
    cudaStream_t st = stream ? (cudaStream_t)stream : b->probs[0]->stream;
    for (int p = 0; p < np; ++p) {
        int rc = ensure_remap_tables(b->probs[p], nullptr);
        if (!rc) rc = stream_after(st, b->probs[p]->stream);
        if (rc) return rc;
    }
    for (int s = 0; s < nsteps; ++s) {
        std::vector<shd_batch::Key> key(np);
        for (int p = 0; p < np; ++p) {
            shd_ctx *c = b->probs[p];
            int slot = -1, cls = 0, rc;
            rc = is_fp64(c) ? ensure_chi_rest<double>(c, st) : ensure_chi_rest<float>(c, st);
            if (rc) return fail(rc, "problem %d: %s", p, std::string(g_err).c_str());
            rc = is_fp64(c) ? graph_slot<double>(c, slot) : graph_slot<float>(c, slot);
            if (rc) return fail(rc, "problem %d: %s", p, std::string(g_err).c_str());
            if (slot < 0) {
                // direct launches for this problem's step
                rc = is_fp64(c) ? run_steps<double>(c, 1, st, false) : run_steps<float>(c, 1, st, false);
                if (rc) return fail(rc, "problem %d: %s", p, std::string(g_err).c_str());
            } else if (b->sweep_mode == 1 && (cls = sweep_batch_class(c)) != 0) {
                int ns = -1;
                rc = capture_presweep<float>(c, &ns);
                if (rc) return fail(rc, "problem %d: %s", p, std::string(g_err).c_str());
                if (ns >= 0) slot = ns;
                else cls = 0;
            }
            key[p] = {c->graph_gen, slot, cls};
        }
        bool any = false;
        for (auto &k : key) any |= k.slot >= 0;
        if (any) {
            const shd_batch::Entry *ent = nullptr;
            for (auto &e : b->cache)
                if (e.key == key) ent = &e;
            if (!ent) {
                if (b->cache.size() >= 8) batch_drop(b);  // problems changed: start over
                shd_batch::Entry fresh;
                fresh.key = key;
                int rc = batch_build(b, key, fresh);
                if (rc) return rc;
                b->cache.push_back(fresh);
                ent = &b->cache.back();
            }
            CK(cudaGraphLaunch(ent->exec, st), "batch graph launch");
            count_launches(ent->extra);
            for (int p = 0; p < np; ++p) {
                if (key[p].slot < 0) continue;
                shd_ctx *c = b->probs[p];
                count_launches(key[p].cls ? c->graph_ns_kernels[key[p].slot] : c->graph_kernels[key[p].slot]);
                std::swap(c->d_Sp, c->d_Sprev);
            }
        }
    }
    for (int p = 0; p < np; ++p) {
        int rc = stream_after(b->probs[p]->stream, st);
        if (rc) return rc;
    }
    return SHD_OK;
}

int shd_batch_set_sweep_mode(shd_batch *b, int mode)
{
    if (!b) return fail(SHD_ERR_ARG, "null batch");
    if (mode != 0 && mode != 1) return fail(SHD_ERR_ARG, "sweep mode %d (0 or 1)", mode);
    if (mode != b->sweep_mode) {
        CK(cudaSetDevice(b->device), "cudaSetDevice");
        CK(cudaDeviceSynchronize(), "synchronize");
        batch_drop(b);
        b->sweep_mode = mode;
    }
    return SHD_OK;
}

void shd_batch_destroy(shd_batch *b)
{
    if (!b) return;
    cudaSetDevice(b->device);
    cudaDeviceSynchronize();
    batch_drop(b);
    delete b;
}

}  // extern "C"
