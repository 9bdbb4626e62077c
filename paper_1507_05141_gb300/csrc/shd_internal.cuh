// Internal declarations of the GB300 SHDOM library: context, device tables,
// device helpers shared by the kernels, and the kernel launchers.
//
// Device layouts
//   discrete-ordinate arrays (I, eta_lab, chi_lab, full boundary):
//     [k][g][o]  with o the node offset in the ordinate's *sweep layout*:
//     the axis the ordinate crosses first (its dominant axis d) is the
//     slowest index, so that every plane normal to d is one contiguous block:
//       d = z : o = (iz*ny + iy)*nx + ix
//       d = y : o = (iy*nz + iz)*nx + ix
//       d = x : o = (ix*nz + iz)*ny + iy
//   spherical-harmonic arrays (I_lm, S_lm): [c][g][p]
//   moments: [c][g][10] = J, H_x, H_y, H_z, K_xx, K_yy, K_zz, K_xy, K_xz, K_yz
#pragma once

#include <cuda_runtime.h>
#include <stdint.h>

#include <string>
#include <vector>

#include "../../include/shdom_gb300.h"

namespace shd {

constexpr double kPi = 3.14159265358979323846;

// temperature grid of the thermal Compton kernel: theta_i = 10^(kThermalLg0 +
// i kThermalDlg), i < kThermalN; nodes blend their two bracketing tables
// linearly in log10(theta) (clamped into the grid)
constexpr double kThermalLg0 = -3.0, kThermalDlg = 0.25;
constexpr int kThermalN = 13;
// nodes per chunk of the thermal source pass (all of one bracket)
constexpr int kThermalChunk = 1024;

// Per-ordinate constants, built on the host in FP64 (Sec. 2.2 mesh; the
// sweep geometry of the short characteristic).
struct Ordinate {
    double n[3];     // direction
    double W;        // quadrature weight (sum 4 pi)
    double fr1, fr2; // upwind-point offsets on the two in-plane axes, in cells
    double s;        // path length from the upwind face to the node
    int d, e1, e2;   // dominant axis and in-plane axes (layout order)
    int sd, s1, s2;  // signs of n along d, e1, e2 (-1, 0, +1)
    int ring, phi;   // (a, b) mesh indices
};

// An 8 x 8 brick of nodes in (x, y) at one z (the unit of the transform
// kernels); flags bit 0: the brick holds at least one moving node.
struct TileInfo {
    int x0, y0, z, flags;
};

// Everything a kernel needs about the problem, passed by value.
template <class T>
struct Prob {
    int nx, ny, nz;
    long long Nc;
    int N, nmu, nphi, NLM, L, G;
    T kappa;
    const Ordinate *ord;   // [N]
    const T *W;            // [N]
    const T *dirs;         // [N][3]
    const T *Y;            // [N][NLM]
    const T *mu;           // [nmu]
    const double *edges;   // [G+1]
    const double *centre;  // [G]
    const T *alpha0;       // [Nc][G]
    const T *ne;           // [Nc]
    const T *u;            // [Nc][3]
    const T *emis0;        // [Nc][G]
    const T *chi0;         // [Nc][G]  alpha0 + ne sigma_out
    const T *K;            // [L+1][G][G]
    const T *sigma_out;    // [G]
    int bc_mode;
    const T *bc;           // ISO: [G]; FULL: DO layout
    const TileInfo *tiles; // [ntiles]
    long long ntiles;
    const long long *moving;      // [nmoving] node ids with u != 0, brick by brick
    long long nmoving;
    const unsigned char *mflag;   // [Nc] 1 where u != 0
    const int *midx;              // [Nc] index of the node in `moving`, -1 at rest
    const int *mtiles;            // [nmtiles] tiles holding a moving node
    long long nmtiles;
    const T *Bproj;        // [N][NB]: W_k Y_p(n_k) | W_k {1, n, nn}/(4 pi) | 0
    int NB;
    int fp64_boost;        // Doppler factor and aberration in FP64 where Gamma > 10
    const int *int2mesh;   // [N] mesh index (a*nphi + b) of internal ordinate k
    const int *mesh2int;   // [N] inverse
    int nA;                // internal ordinates [0, nA) cross z or y first, [nA, N) x
    const T *lc;           // [G] log of the group centres
    const T *linv;         // [G] 1/(lc[g+1] - lc[g])
    T le0, leG;            // log of the outer edges
    int lgu;               // group centres equally spaced in log energy; then
    T lgidl;               // 1 / that spacing,
    T lgx0, lgx1;          // the outer edges in units of it, from lc[0]
    // thermal electrons (SHD_SCAT_KN_THERMAL): per node its bracket on the
    // temperature grid and the weight of the upper table; the kernels and
    // out-scattering cross-sections on the grid; nodes grouped by bracket
    int thermal;
    const int *thb;        // [Nc]
    const T *thw;          // [Nc]
    const T *thK;          // [kThermalN][L+1][G][G]
    const T *thso;         // [kThermalN][G]
    const int *thperm;     // [Nc] node ids ordered by bracket
    const int4 *thchunk;   // {first index into thperm, count, bracket, 0}
    int nthchunk;
};

// Per-stage CUDA events recorded on the launching stream without any host
// synchronisation; read (and summed) only by shd_get_timing.
struct Timing {
    static constexpr int kStages = 5;  // project, source, sums, sh2lab, sweep
    static constexpr int kCap = 2048;  // steps recorded per enable
    bool on = false;
    std::vector<cudaEvent_t> pool;     // (kStages + 1) per recorded step
    long long count = 0;               // steps recorded
};

}  // namespace shd

struct shd_ctx {
    int device = 0;
    int precision = SHD_FP64;
    size_t esize = 8;  // bytes per real on the device
    cudaStream_t stream = nullptr;

    // grid
    int nx = 0, ny = 0, nz = 0;
    double lx = 0, ly = 0, lz = 0, h[3] = {0, 0, 0};
    long long Nc = 0;
    // angles
    int L = -1, nmu = 0, nphi = 0, N = 0, NLM = 0;
    // host tables (FP64).  *_mesh are in mesh order k = a*nphi + b; the others
    // in the internal order, which groups the ordinates by the axis they cross
    // first (z, then y, then x) so that each group shares one sweep layout
    std::vector<double> h_mu, h_wmu, h_dirs, h_W, h_Y;
    std::vector<double> h_dirs_mesh, h_W_mesh, h_Y_mesh;
    std::vector<int> h_int2mesh, h_mesh2int;
    int nA = 0;  // internal ordinates crossing z or y first
    int nZ = 0;  // internal ordinates crossing z first ([0, nZ))
    int *d_int2mesh = nullptr, *d_mesh2int = nullptr;
    std::vector<shd::Ordinate> h_ord;
    // groups
    int G = 0;
    std::vector<double> h_edges, h_centre;
    bool lg_uniform = false;       // centres equally spaced in log energy
    double lg_dl = 1.0, lg_c0 = 0; // that spacing, the first log centre

    bool have_grid = false, have_angles = false, have_groups = false;
    bool have_fields = false, have_scat = false, have_state = false;
    int scat_kind = 0;
    bool k_diagonal = false;  // every K_l[g][g'] is zero off the diagonal
    int bc_mode = SHD_BC_VACUUM;
    double kappa = 0.0;

    // device buffers (reals are T = double or float per precision)
    void *d_ord = nullptr;
    void *d_W = nullptr, *d_dirs = nullptr, *d_Y = nullptr, *d_mu = nullptr;
    double *d_edges = nullptr, *d_centre = nullptr;
    void *d_alpha0 = nullptr, *d_ne = nullptr, *d_u = nullptr, *d_emis0 = nullptr, *d_chi0 = nullptr;
    // host maxima of the fields and of sigma_out: a bound on the optical depth
    // of one short-characteristic step (the sweep's FP64 weights)
    double h_alpha_max = 0, h_ne_max = 0, h_gamma_max = 1, h_sigma_max = 0;
    // chi0 in the three sweep layouts [d][g][o] and, per layout, the 4-node
    // pieces of each plane holding a moving node: bit (id % 64) of
    // d_mbits[d][id / 64][piece] (mbits_nwin windows of mbits_npc words)
    void *d_chi0L = nullptr;
    unsigned long long *d_mbits = nullptr;
    int mbits_npc = 0, mbits_nwin = 0;
    void *d_K = nullptr, *d_sigma_out = nullptr;
    void *d_bc = nullptr;
    void *d_I = nullptr, *d_eta = nullptr, *d_chi = nullptr;
    void *d_Ip = nullptr, *d_Sp = nullptr, *d_Sprev = nullptr, *d_mom = nullptr;
    double *d_sums = nullptr;     // [3] energy, photons, resid
    double *d_partial = nullptr;  // reduction scratch
    int n_partial = 0;
    void *d_tiles = nullptr;          // TileInfo[ntiles]
    long long ntiles = 0;
    long long *d_moving = nullptr;    // moving node ids
    long long nmoving = 0;
    unsigned char *d_mflag = nullptr; // [Nc]
    // device staging of the fields as given (FP64) and the result of their check
    void *d_fstage = nullptr;
    size_t fstage_n = 0;
    void *d_fcheck = nullptr;
    void *d_Bproj = nullptr;          // [N][NB]
    int NB = 0;
    int *d_midx = nullptr;            // [Nc] moving index or -1
    int *d_mtiles = nullptr;          // tiles holding a moving node
    long long nmtiles = 0;
    // node-major scratch [m][g][k] of the moving nodes (Lorentz remaps):
    // project: nm[0] = laboratory I, nm[1] = comoving I0;
    // sh2lab:  nm[0] = comoving S0, nm[1] = eta_lab, nm[2] = chi_lab
    void *d_nm[3] = {nullptr, nullptr, nullptr};
    // FP32 remap tables of the moving nodes, [m][k] float4 {stencil code,
    // t, tp, Doppler ratio}: [0] comoving remap (n_k boosted to the
    // laboratory, nu/nu0), [1] laboratory remap (n_k boosted to the comoving
    // frame, nu0/nu); rebuilt after the fields or angles change
    void *d_rtab[2] = {nullptr, nullptr};
    unsigned short *d_rrng[2] = {nullptr, nullptr};  // FP64-decided in-range output groups of the remap tables
    void *d_dirs64 = nullptr;                         // internal-order directions in FP64
    bool fstage_u_current = false;                    // the staging area holds the flow in use
    size_t rtab_n = 0;
    bool rtab_valid = false;
    void *d_lc = nullptr, *d_linv = nullptr;  // log-energy group tables
    // tensor-core operands of the mixed path (BF16 hi / lo, canonical K-major)
    void *d_tc_Bh = nullptr, *d_tc_Bl = nullptr;  // [NB][tc_Kp]   projection matrix
    void *d_tc_Yh = nullptr, *d_tc_Yl = nullptr;  // [tc_Np][tc_Kq] harmonics
    int tc_Kp = 0, tc_Np = 0, tc_Kq = 0;
    int *d_tc_err = nullptr;                      // set by a kernel whose wait timed out
    // BF16 hi / lo of the scattering kernel K_l for the tensor-core source
    // (MIXED with a kernel that mixes groups): [2][L+1][Gp][Kp]
    void *d_tcK = nullptr;
    // source pass of such a kernel in MIXED: 0 not timed yet, 1 CUDA cores,
    // 2 tensor cores (the faster when first timed: source_ms = {CUDA-core,
    // tensor-core} milliseconds)
    int source_choice = 0;
    float source_ms[2] = {0.f, 0.f};
    // segment tiling of the mixed path: group 0 = z- and y-class ordinates
    // over bw x (128/bw) boxes of (x, y) at one z; group 1 = x-class over
    // boxes of (y, z) at one x.  Segments {plane, a0, b0, 0}; the group's
    // ordinates in slots (each class padded to a multiple of 32) with the
    // operands over slots (BF16 hi / lo, canonical K-major) and per chunk of
    // 32 slots {class map index in the group, first ordinate of the chunk in
    // its class, internal index of the class's first ordinate, class size}
    void *d_seg[2] = {nullptr, nullptr};
    long long nseg[2] = {0, 0};
    int seg_bw[2] = {0, 0};
    void *d_tcs_Bh[2] = {nullptr, nullptr}, *d_tcs_Bl[2] = {nullptr, nullptr};  // [NB][tcs_Kp]
    void *d_tcs_Yh[2] = {nullptr, nullptr}, *d_tcs_Yl[2] = {nullptr, nullptr};  // [tcs_Kp][tc_Kq]
    int tcs_Kp[2] = {0, 0}, tcs_nchunk[2] = {0, 0};
    int tcs_chunk[2][16][4] = {};
    bool seg_ready = false;
    double *d_stage = nullptr;    // staging buffer for host <-> device copies (FP64)
    size_t stage_elems = 0;
    long long bytes = 0;
    bool sprev_valid = false;

    // schedule of the FP32 plane sweep: planes split over clusters of
    // sweep_C CTAs of sweep_NT threads (0 = not chosen yet).  Forced by
    // shd_set_sweep_schedule, else chosen by timing the schedules that fit on
    // the first sweep launched outside a stream capture (sweep_tune: C, NT
    // and milliseconds of each candidate); dropped when the sizes change
    int sweep_force_C = 0, sweep_force_NT = 0;
    int sweep_C = 0, sweep_NT = 0;
    int sweep_ntune = 0;
    float sweep_tune[16][3] = {};

    // Ng acceleration of shd_solve_static (0: off; else the period >= 4):
    // the last three source iterates and the inner-product scratch
    int ng_period = 0;
    void *d_ng[3] = {nullptr, nullptr, nullptr};
    double *d_ngpart = nullptr;  // [kNgBlocks * 5 + 5]
    // time scheme of shd_step (SHD_TIME_EULER / SHD_TIME_RK4) and the three
    // discrete-ordinate arrays of the Runge-Kutta sub-steps: I(t), the
    // sub-solve input, the sum of increments; plus the saved sums
    int time_scheme = SHD_TIME_EULER;
    // source interpolation of the sweep (SHD_SC_LINEAR / SHD_SC_BEZIER)
    int integrator = SHD_SC_LINEAR;
    // thermal electrons: the node temperatures as given (host, FP64), their
    // brackets and weights, the nodes grouped by bracket, the kernels on the
    // temperature grid in the working precision
    bool have_theta = false;
    std::vector<double> h_theta;
    int *d_thb = nullptr, *d_thperm = nullptr;
    void *d_thw = nullptr, *d_thK = nullptr, *d_thso = nullptr;
    int4 *d_thchunk = nullptr;
    int nthchunk = 0;
    void *d_rk[3] = {nullptr, nullptr, nullptr};
    double *d_sums_save = nullptr;  // [2]

    shd::Timing timing;

    // one time step captured as a CUDA graph per parity of the S_lm / S_prev
    // pair (graph_sp[i]: the buffer that step writes S_lm to); dropped by
    // every setter, rebuilt on the next step
    cudaGraph_t graph[2] = {nullptr, nullptr};
    cudaGraphExec_t gexec[2] = {nullptr, nullptr};
    unsigned long long graph_gen = 0;  // bumped whenever a graph is captured or dropped
    // the step without its sweep, per S_lm buffer (graph_ns_sp[i]), for a
    // batch that sweeps its problems in one launch; captured on demand and
    // dropped with the graphs
    cudaGraph_t graph_ns[2] = {nullptr, nullptr};
    void *graph_ns_sp[2] = {nullptr, nullptr};
    unsigned long long graph_ns_kernels[2] = {0, 0};
    bool skip_sweep = false;  // set only while the sweep-less step is captured
    // chi_lab at the nodes at rest against chi0 (k_chi_rest_fill), so that a3
    // need not store it every step: 0 it holds chi0; 1 it holds chi0 unless
    // the device word d_chi_dirty says chi0 changed since the last fill
    // (k_chi0_layout raises it); 2 it must be filled (new buffers or moving set)
    int chi_rest_state = 2;
    int *d_chi_dirty = nullptr;
    void *graph_sp[2] = {nullptr, nullptr};
    unsigned long long graph_kernels[2] = {0, 0};  // kernel launches per replay
    cudaStream_t cap_stream = nullptr;
    bool graphs_off = false;  // a capture failed: launch directly from then on
};

namespace shd {

// Counts a kernel launch issued by the library (see shd_launch_count).
void note_launch();

// SHD_OK when ctx can run a step: configured, and every stage's shared
// memory within the limit (else the code, with the message in shd_last_error).
int check_ready(shd_ctx *ctx);

// -------------------------------------------------------------------------
// device helpers
// -------------------------------------------------------------------------

__host__ __device__ inline long long perm_offset(int d, int ix, int iy, int iz, int nx, int ny, int nz)
{
    if (d == 2) return ((long long)iz * ny + iy) * nx + ix;
    if (d == 1) return ((long long)iy * nz + iz) * nx + ix;
    return ((long long)ix * nz + iz) * ny + iy;
}

template <class T>
__device__ inline T dsqrt(T x);
template <>
__device__ inline double dsqrt<double>(double x) { return sqrt(x); }
template <>
__device__ inline float dsqrt<float>(float x) { return sqrtf(x); }

template <class T>
__device__ inline T dexp(T x);
template <>
__device__ inline double dexp<double>(double x) { return exp(x); }
template <>
__device__ inline float dexp<float>(float x) { return expf(x); }

template <class T>
__device__ inline T dlog(T x);
template <>
__device__ inline double dlog<double>(double x) { return log(x); }
template <>
__device__ inline float dlog<float>(float x) { return logf(x); }

// Rounding and clamping in the argument's own precision: on GB300 a float
// taken through double runs on the FP64 pipe, dozens of times slower.
template <class T>
__device__ inline T dfloor(T x);
template <>
__device__ inline double dfloor<double>(double x) { return ::floor(x); }
template <>
__device__ inline float dfloor<float>(float x) { return floorf(x); }

template <class T>
__device__ inline T dabs(T x);
template <>
__device__ inline double dabs<double>(double x) { return ::fabs(x); }
template <>
__device__ inline float dabs<float>(float x) { return fabsf(x); }

template <class T>
__device__ inline T dclamp(T x, T lo, T hi);
template <>
__device__ inline double dclamp<double>(double x, double lo, double hi) { return ::fmin(::fmax(x, lo), hi); }
template <>
__device__ inline float dclamp<float>(float x, float lo, float hi) { return fminf(fmaxf(x, lo), hi); }

template <class T>
__device__ inline T datan2(T y, T x);
template <>
__device__ inline double datan2<double>(double y, double x) { return atan2(y, x); }
template <>
__device__ inline float datan2<float>(float y, float x) { return atan2f(y, x); }

// Lorentz boost of a direction (Sec. 2.2, eq:lorentzfreq and eq:lorentzray
// with u = Gamma v/c).  sgn = +1: laboratory n -> comoving, returning
// nu0/nu = Gamma - u.n;  sgn = -1: comoving n -> laboratory, returning
// nu/nu0 = Gamma + u.n.  The ratio is formed as 1/(Gamma+|u|) + |u||n -+ u^|^2/2,
// free of cancellation at large Gamma.
template <class R>
__device__ inline R boost_dir(const R u[3], const R n[3], R out[3], R sgn)
{
    R uu = u[0] * u[0] + u[1] * u[1] + u[2] * u[2];
    R gam = dsqrt<R>(R(1) + uu), um = dsqrt<R>(uu);
    if (!(um > R(0))) {  // at rest (or |u|^2 underflowed): the identity
        out[0] = n[0]; out[1] = n[1]; out[2] = n[2];
        return R(1);
    }
    R un = u[0] * n[0] + u[1] * n[1] + u[2] * n[2];
    R d2 = 0;
    if constexpr (sizeof(R) == 4) {
        // single precision: one reciprocal of |u| serves the three components
        const R ium = R(1) / um;
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            R dd = n[i] - sgn * (u[i] * ium);
            d2 += dd * dd;
        }
    } else {
#pragma unroll
        for (int i = 0; i < 3; ++i) {
            R dd = n[i] - sgn * u[i] / um;
            d2 += dd * dd;
        }
    }
    R r = R(1) / (gam + um) + R(0.5) * um * d2;
    R f = R(1) - sgn * un / (gam + R(1));
    R ir = R(1) / r;
#pragma unroll
    for (int i = 0; i < 3; ++i) out[i] = (n[i] - sgn * u[i] * f) * ir;
    return r;
}

// The boost of boost_dir evaluated in FP64 for a float problem (the mixed
// path's FP64 island for Lorentz factors above 10).
__device__ inline float boost_dir_fp64(const float u[3], const float n[3], float out[3], float sgn)
{
    double ud[3] = {u[0], u[1], u[2]}, nd[3] = {n[0], n[1], n[2]}, od[3];
    double r = boost_dir<double>(ud, nd, od, (double)sgn);
    out[0] = (float)od[0]; out[1] = (float)od[1]; out[2] = (float)od[2];
    return (float)r;
}

template <class T>
__device__ inline T boost_any(const T u[3], const T n[3], T out[3], T sgn, int fp64_boost)
{
    return boost_dir<T>(u, n, out, sgn);
}
template <>
__device__ inline float boost_any<float>(const float u[3], const float n[3], float out[3], float sgn, int fp64_boost)
{
    if (fp64_boost && u[0] * u[0] + u[1] * u[1] + u[2] * u[2] > 99.f) return boost_dir_fp64(u, n, out, sgn);
    return boost_dir<float>(u, n, out, sgn);
}

// Bilinear stencil on an ordinate mesh (mu ascending Gauss rings, phi
// uniform from 0): four (ordinate, weight) pairs plus an optional pole term
// whose value is the average of ring `pole_ring`.
template <class T>
struct Stencil {
    int k[4];
    T w[4];
    int pole_ring;  // -1: none
    T wpole;
};

// The stencil's placement on the mesh: between rings a and a+1 (mode 0),
// between a pole and its outer ring a (1 south, 2 north), or on the single
// ring of a one-ring mesh (3); phi bin b; fractions t (mu) and tp (phi).
template <class T>
struct StencilParams {
    int mode, a, b;
    T t, tp;
};

template <class T>
__device__ inline StencilParams<T> stencil_params(const T *mu, int nmu, int nphi, const T n[3])
{
    StencilParams<T> p;
    T m = n[2];
    m = m > T(1) ? T(1) : (m < T(-1) ? T(-1) : m);
    T phi = datan2<T>(n[1], n[0]);
    if (phi < T(0)) phi += T(2 * kPi);
    T x = phi * (T(nphi) / T(2 * kPi));
    int b = (int)x;  // x >= 0
    T tp = x - T(b);
    if (b >= nphi) b -= nphi;
    if (!(b >= 0 && b < nphi)) { b = 0; tp = 0; }  // non-finite direction: stay in bounds
    p.b = b;
    p.tp = tp;
    if (m < mu[0] || m > mu[nmu - 1]) {
        const bool south = m < mu[0];
        p.mode = south ? 1 : 2;
        p.a = south ? 0 : nmu - 1;
        p.t = south ? (m + T(1)) / (mu[0] + T(1)) : (T(1) - m) / (T(1) - mu[nmu - 1]);
        return p;
    }
    if (nmu > 1) {
        // ring bracket: the largest a <= nmu - 2 with mu[a] < m (0 if none),
        // by bisection over the ascending nodes
        int a = 0, hi = nmu - 2;
        while (a < hi) {
            const int mid = (a + hi + 1) >> 1;
            if (mu[mid] < m) a = mid;
            else hi = mid - 1;
        }
        p.mode = 0;
        p.a = a;
        p.t = (m - mu[a]) / (mu[a + 1] - mu[a]);
    } else {
        p.mode = 3;
        p.a = 0;
        p.t = 0;
    }
    return p;
}

// Four (mesh ordinate, weight) pairs plus the pole term of a placement.
template <class T>
__device__ inline Stencil<T> stencil_from_params(const StencilParams<T> &p, int nphi)
{
    Stencil<T> s;
    const int b = p.b, b1 = b + 1 == nphi ? 0 : b + 1;
    const T t = p.t, tp = p.tp;
    s.pole_ring = -1;
    s.wpole = 0;
    if (p.mode == 1 || p.mode == 2) {
        const int ring = p.a;
        s.pole_ring = ring;
        s.wpole = T(1) - t;
        s.k[0] = ring * nphi + b;  s.w[0] = t * (T(1) - tp);
        s.k[1] = ring * nphi + b1; s.w[1] = t * tp;
        s.k[2] = s.k[0]; s.w[2] = 0;
        s.k[3] = s.k[1]; s.w[3] = 0;
    } else if (p.mode == 0) {
        const int a = p.a;
        s.k[0] = a * nphi + b;       s.w[0] = (T(1) - t) * (T(1) - tp);
        s.k[1] = a * nphi + b1;      s.w[1] = (T(1) - t) * tp;
        s.k[2] = (a + 1) * nphi + b; s.w[2] = t * (T(1) - tp);
        s.k[3] = (a + 1) * nphi + b1; s.w[3] = t * tp;
    } else {
        s.k[0] = b; s.w[0] = T(1) - tp;
        s.k[1] = b1; s.w[1] = tp;
        s.k[2] = b; s.w[2] = 0;
        s.k[3] = b1; s.w[3] = 0;
    }
    return s;
}

template <class T>
__device__ inline Stencil<T> make_stencil(const T *mu, int nmu, int nphi, const T n[3])
{
    return stencil_from_params<T>(stencil_params<T>(mu, nmu, nphi, n), nphi);
}

// F points at one group's N ordinate values; poles at that group's two ring
// averages (south, north).
template <class T>
__device__ inline T eval_stencil(const Stencil<T> &s, const T *F, const T *poles)
{
    T v = s.w[0] * F[s.k[0]] + s.w[1] * F[s.k[1]] + s.w[2] * F[s.k[2]] + s.w[3] * F[s.k[3]];
    if (s.pole_ring >= 0) v += s.wpole * poles[s.pole_ring == 0 ? 0 : 1];
    return v;
}

// Group bracket for an energy, in log energy (Sec. 2.3 multi-group; the group
// value is taken at the centre).  lc[g] = log centre, inv[g] = 1/(lc[g+1] -
// lc[g]), le0 / leG = log of the outer edges.  Modes: 0 outside the edges
// (ga = nearest group), 1 a single group ga (between an outer centre and its
// edge), 2 between centres ga and ga+1 with fraction t in log energy.
template <class T>
struct FreqBracket {
    int mode, ga;
    T t;
};

// `hint` is a lower bound for the bracket index carried between calls with
// non-decreasing energies; the search moves forward from it.
template <class T>
__device__ inline FreqBracket<T> freq_bracket(const T *lc, const T *inv, T le0, T leG, int G, T le, int &hint)
{
    FreqBracket<T> b;
    b.t = T(0);
    if (le < le0 || le > leG) { b.mode = 0; b.ga = le < le0 ? 0 : G - 1; return b; }
    if (le <= lc[0]) { b.mode = 1; b.ga = 0; return b; }
    if (le >= lc[G - 1]) { b.mode = 1; b.ga = G - 1; return b; }
    int lo = hint < 0 ? 0 : (hint > G - 2 ? G - 2 : hint);
    if (lc[lo] > le) lo = 0;
    while (lo < G - 2 && lc[lo + 1] <= le) ++lo;
    hint = lo;
    b.mode = 2;
    b.ga = lo;
    b.t = (le - lc[lo]) * inv[lo];
    return b;
}

// Single-precision hardware approximations (PTX .approx.ftz: subnormal
// arguments and results are flushed to zero): 2^x, log2(x), 1/x.
__device__ inline float hw_exp2(float x)
{
    float y;
    asm("ex2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ inline float hw_log2(float x)
{
    float y;
    asm("lg2.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
__device__ inline float hw_rcp(float x)
{
    float y;
    asm("rcp.approx.ftz.f32 %0, %1;" : "=f"(y) : "f"(x));
    return y;
}
constexpr float kLog2eF = 1.44269504088896341f;  // 1/ln 2

// Geometric between positive values, linear in log(eps) otherwise.
template <class T>
__device__ inline T freq_mix(T fa, T fb, T t);
template <>
__device__ inline double freq_mix<double>(double fa, double fb, double t)
{
    if (fa > 0.0 && fb > 0.0) return fa * exp(t * log(fb / fa));
    return (1.0 - t) * fa + t * fb;
}
template <>
__device__ inline float freq_mix<float>(float fa, float fb, float t)
{
    // fa^(1-t) fb^t = fa 2^(t log2(fb/fa)) by the hardware approximations
    // while every operand stays a normal number, else by the library
    if (fa >= 1.17549435e-38f && fb >= 1.17549435e-38f) {
        const float r = fb * hw_rcp(fa);
        if (r >= 1.17549435e-38f && r <= 3.4e38f) return fa * hw_exp2(t * hw_log2(r));
    }
    if (fa > 0.f && fb > 0.f) return fa * expf(t * logf(fb / fa));
    return (1.f - t) * fa + t * fb;
}

// Geometric mix whose log ratio lr = log2(fb/fa) is already known (both
// positive).
template <class T>
__device__ inline T freq_mix_lr(T fa, T lr, T t);
template <>
__device__ inline double freq_mix_lr<double>(double fa, double lr, double t)
{
    return fa * exp2(t * lr);
}
template <>
__device__ inline float freq_mix_lr<float>(float fa, float lr, float t)
{
    return fa * hw_exp2(t * lr);
}

// Linear-in-tau short-characteristic weights with e = exp(-x):
//   I_P = I_U e + S_P wp + S_U wu,  wp = 1 - (1-e)/x,  wu = (1-e)/x - e.
// Below the threshold the Taylor series (Horner) avoids the cancellation;
// its coefficients are constants folded at compile time (a division by a
// constant would be a full division sequence on every update).
template <class T>
__device__ inline void sc_weights(T x, T &e, T &wp, T &wu);

template <>
__device__ inline void sc_weights<double>(double x, double &e, double &wp, double &wu)
{
    if (x < 0.05) {
        // wp = sum_{n>=1} (-1)^{n+1} x^n/(n+1)!,  wu = sum_{n>=1} (-1)^{n+1} n x^n/(n+1)!
        wp = x * (1.0 / 2 - x * (1.0 / 6 - x * (1.0 / 24 - x * (1.0 / 120 - x * (1.0 / 720 - x * (1.0 / 5040 - x * (1.0 / 40320 - x * (1.0 / 362880.0))))))));
        wu = x * (1.0 / 2 - x * (1.0 / 3 - x * (1.0 / 8 - x * (1.0 / 30 - x * (1.0 / 144 - x * (1.0 / 840 - x * (1.0 / 5760 - x * (1.0 / 45360.0))))))));
        e = exp(-x);
        return;
    }
    double em1 = -expm1(-x);
    e = 1.0 - em1;
    double a0 = em1 / x;
    wp = 1.0 - a0;
    wu = a0 - e;
}

// Above this optical depth the single-precision exponential loses more than
// ~1e-6 relative accuracy (its argument carries x times the rounding of the
// scaling): the weights are then taken in FP64.
constexpr float kFp64Tau = 16.f;

// The weights in working precision only: for sweeps whose optical depth per
// step is bounded by kFp64Tau on the host (see the sweep launcher).
template <class T>
__device__ inline void sc_weights_narrow(T x, T &e, T &wp, T &wu);

template <>
__device__ inline void sc_weights_narrow<double>(double x, double &e, double &wp, double &wu)
{
    sc_weights<double>(x, e, wp, wu);
}

// The same weights with the two series of the small-x branch advanced
// together by packed FP32 instructions (lane 0 wp, lane 1 wu; each lane
// rounds exactly as the scalar fused multiply-add does).
__device__ inline void sc_weights_narrow_x2(float x, float &e, float &wp, float &wu)
{
    e = hw_exp2(-x * kLog2eF);
    if (x < 0.5f) {
        const float2 nx = make_float2(-x, -x);
        float2 a = __ffma2_rn(nx, make_float2(1.f / 362880.f, 1.f / 45360.f), make_float2(1.f / 40320, 1.f / 5760));
        a = __ffma2_rn(nx, a, make_float2(1.f / 5040, 1.f / 840));
        a = __ffma2_rn(nx, a, make_float2(1.f / 720, 1.f / 144));
        a = __ffma2_rn(nx, a, make_float2(1.f / 120, 1.f / 30));
        a = __ffma2_rn(nx, a, make_float2(1.f / 24, 1.f / 8));
        a = __ffma2_rn(nx, a, make_float2(1.f / 6, 1.f / 3));
        a = __ffma2_rn(nx, a, make_float2(1.f / 2, 1.f / 2));
        a = __fmul2_rn(make_float2(x, x), a);
        wp = a.x;
        wu = a.y;
        return;
    }
    float a0 = (1.f - e) * hw_rcp(x);
    wp = 1.f - a0;
    wu = a0 - e;
}

template <>
__device__ inline void sc_weights_narrow<float>(float x, float &e, float &wp, float &wu)
{
    e = hw_exp2(-x * kLog2eF);
    if (x < 0.5f) {
        wp = x * (1.f / 2 - x * (1.f / 6 - x * (1.f / 24 - x * (1.f / 120 - x * (1.f / 720 - x * (1.f / 5040 - x * (1.f / 40320 - x * (1.f / 362880.f))))))));
        wu = x * (1.f / 2 - x * (1.f / 3 - x * (1.f / 8 - x * (1.f / 30 - x * (1.f / 144 - x * (1.f / 840 - x * (1.f / 5760 - x * (1.f / 45360.f))))))));
        return;
    }
    // x >= 1/2: e <= 0.61, so 1 - e carries no cancellation
    float a0 = (1.f - e) * hw_rcp(x);
    wp = 1.f - a0;
    wu = a0 - e;
}

template <>
__device__ inline void sc_weights<float>(float x, float &e, float &wp, float &wu)
{
    if (x > kFp64Tau) {
        const double xd = x, ed = exp(-xd), a0 = (1.0 - ed) / xd;
        e = (float)ed;
        wp = (float)(1.0 - a0);
        wu = (float)(a0 - ed);
        return;
    }
    sc_weights_narrow<float>(x, e, wp, wu);
}

// Cubic Bezier short characteristic (Sec. 2: the paper's cubic Bezier ray
// tracing): over a segment of optical depth x with end values S_U, S_P and
// control points C_U, C_P,  I_P = I_U e + wU S_U + wCU C_U + wCP C_P + wP S_P,
// the weights being x times the integrals of the cubic Bernstein polynomials
// against e^-(x - t):  with E_k = int_0^1 v^k e^(-x v) dv,  wU = x E3,
// wCU = 3x (E2 - E3), wCP = 3x (E1 - 2 E2 + E3), wP = x (E0 - 3 E1 + 3 E2 - E3).
// Small x: E3 by its power series sum_m (-x)^m / (m! (m + 4)), then the
// stable downward recursion E_(k-1) = (x E_k + e)/k; large x: E0 = (1 - e)/x
// and the upward recursion E_k = (k E_(k-1) - e)/x.
template <class T>
__device__ inline void bezier_weights(T x, T &e, T &wU, T &wCU, T &wCP, T &wP)
{
    T E0, E1, E2, E3;
    constexpr bool F = sizeof(T) == 4;
    e = F ? (T)hw_exp2((float)(-x * kLog2eF)) : (T)exp((double)-x);
    const T xs = F ? T(2) : T(1);
    if (x < xs) {
        constexpr int M = F ? 14 : 24;
        // Horner over m of (-x)^m / (m! (m + 4))
        T acc = T(1) / T(M + 4);
#pragma unroll
        for (int m = M - 1; m >= 0; --m) acc = T(1) / T(m + 4) - x * acc / T(m + 1);
        E3 = acc;
        E2 = (x * E3 + e) / T(3);
        E1 = (x * E2 + e) / T(2);
        E0 = x * E1 + e;
    } else {
        E0 = (T(1) - e) / x;
        E1 = (E0 - e) / x;
        E2 = (T(2) * E1 - e) / x;
        E3 = (T(3) * E2 - e) / x;
    }
    wU = x * E3;
    wCU = T(3) * x * (E2 - E3);
    wCP = T(3) * x * (E1 - T(2) * E2 + E3);
    wP = x * (E0 - T(3) * E1 + T(3) * E2 - E3);
}

// Derivative of the source along the ray at a node from its upwind and
// downwind slopes du, dd over optical depths xu, xd: Fritsch and Butland's
// weighted harmonic mean du dd / (a dd + (1 - a) du), a = (1 + xd/(xu+xd))/3,
// when du and dd have the same sign, else 0.
template <class T>
__device__ inline T fb_derivative(T du, T dd, T xu, T xd)
{
    if (!(du * dd > T(0))) return T(0);
    const T a = (T(1) + xd / (xu + xd)) / T(3);
    return du * dd / (a * dd + (T(1) - a) * du);
}

// -------------------------------------------------------------------------
// launchers (shd_kernels.cu)
// -------------------------------------------------------------------------
template <class T>
Prob<T> make_prob(const shd_ctx *ctx);

template <class T>
cudaError_t launch_chi0(const shd_ctx *ctx, cudaStream_t st);
template <class T>
cudaError_t launch_project(const shd_ctx *ctx, const T *I, T *Ip, T *mom, cudaStream_t st);
template <class T>
cudaError_t launch_project_scratch(const shd_ctx *ctx, const T *I, T *Ip, T *mom, T *scratch, cudaStream_t st);
bool tc_usable(const shd_ctx *ctx);
bool seg_usable(const shd_ctx *ctx);
bool seg_manual(const shd_ctx *ctx);
cudaError_t launch_project_seg(const shd_ctx *ctx, const float *I, float *Ip, float *mom, float *nm0, float *nm1,
                               cudaStream_t st);
cudaError_t launch_sh2lab_seg(const shd_ctx *ctx, const float *Sp, float *eta, float *chi, float *nm0, float *nm1,
                              float *nm2, cudaStream_t st, bool full_chi);
cudaError_t launch_remap_tables_f(const shd_ctx *ctx, float4 *tc, float4 *tl, unsigned short *rc, unsigned short *rl,
                                  const double *u64, const double *dirs64, cudaStream_t st);
cudaError_t launch_remap_to_comoving_f(const shd_ctx *ctx, const float *nm0, float *nm1, cudaStream_t st);
cudaError_t launch_remap_to_lab_f(const shd_ctx *ctx, const float *nm0, float *nm1, float *nm2, cudaStream_t st);
size_t project_tc_smem_bytes(const shd_ctx *ctx);
size_t sh2lab_tc_smem_bytes(const shd_ctx *ctx);
cudaError_t launch_project_tc(const shd_ctx *ctx, const float *I, float *Ip, float *mom, const float *I0n,
                              cudaStream_t st);
cudaError_t launch_sh2lab_tc(const shd_ctx *ctx, const float *Sp, float *eta, float *chi, float *S0n,
                             cudaStream_t st);
template <class T>
cudaError_t launch_source(const shd_ctx *ctx, const T *Ip, T *Sp, cudaStream_t st);
template <class T>
cudaError_t launch_sh2lab(const shd_ctx *ctx, const T *Sp, T *eta, T *chi, cudaStream_t st, bool full_chi = true);
template <class T>
cudaError_t launch_sweep(const shd_ctx *ctx, T *I, const T *eta, const T *chi, cudaStream_t st,
                         bool use_chi0L = false);
template <class T>
bool sweep_uses_chi0L(const shd_ctx *ctx);
// chi_lab[k][g][o] = chi0L[d(k)][g][o] for every ordinate, group and node
// (the value a3 stores at a node at rest, in the sweep layout)
// force = 0: only if *d_chi_dirty is set; the word is cleared after the fill
template <class T>
cudaError_t launch_chi_rest_fill(const shd_ctx *ctx, T *chi, cudaStream_t st, bool force);
bool sweep_schedule_valid(const shd_ctx *ctx, int C, int NT);

// One problem of a batched plane sweep (k_sweep_batch): its fields, arrays
// and flags, and the first of its items ((ordinate, group) pairs) in the
// batch's work list.
struct SweepBatchProb {
    Prob<float> P;
    float *I;
    const float *eta, *chi, *chi0L;
    const unsigned long long *mbits;
    int npc, nwin, cb, wide;
    long long item0;
};
// The class of the one-CTA plane sweep a batch runs for the problem (U in
// bits 0-2, the chi0 table bit 3, FP64 weights bit 4; problems of one class
// share a launch); 0 when its sweep is not that kernel's (FP64, Bezier,
// planes that are not 16-byte multiples or too large) or when a cluster
// schedule, forced or timed more than 3 % faster, sweeps it.
int sweep_batch_class(const shd_ctx *ctx);
size_t sweep_batch_smem(const shd_ctx *ctx);
void sweep_batch_fill(const shd_ctx *ctx, SweepBatchProb &d, long long item0);
cudaError_t launch_sweep_batch(int cls, const SweepBatchProb *d_probs, int nprob, long long nitems, size_t smem,
                               int device, cudaStream_t st);
bool sweep_bez_usable(const shd_ctx *ctx);
template <class T>
cudaError_t launch_sums(shd_ctx *ctx, const T *mom, const T *Sp, const T *Sprev, bool have_prev, cudaStream_t st);
template <class T>
cudaError_t launch_source_sums(shd_ctx *ctx, const T *Ip, T *Sp, const T *mom, const T *Sprev, bool have_prev,
                               cudaStream_t st);
template <class T>
bool source_sums_usable(const shd_ctx *ctx);

// layout conversions: canonical FP64 [c][g][k] chunk <-> device DO layout
template <class T>
cudaError_t launch_canon_to_do(const shd_ctx *ctx, const double *src, T *dst, long long c0, long long nc,
                               cudaStream_t st);
template <class T>
cudaError_t launch_do_to_canon(const shd_ctx *ctx, const T *src, double *dst, long long c0, long long nc,
                               cudaStream_t st);
template <class T>
cudaError_t launch_convert(const double *src, T *dst, long long n, cudaStream_t st);
template <class T>
cudaError_t launch_convert_back(const T *src, double *dst, long long n, cudaStream_t st);

cudaError_t launch_kn_table(int G, const double *d_edges, int L, double *d_K, double *d_sigma_out,
                            const double *d_gx, const double *d_gw, int nq, cudaStream_t st);
// the thermal Compton kernels on the temperature grid (FP64): quad holds the
// Gauss-Legendre nodes and weights of the electron speed, electron direction,
// scattering cosine and incident energy rules (see k_kn_thermal_table)
cudaError_t launch_kn_thermal_tables(int G, const double *d_edges, int L, const double *d_quad, double *d_K,
                                     double *d_so, cudaStream_t st);
// thermal source pass (a2 + the a5 partials over grid CTAs)
template <class T>
cudaError_t launch_source_thermal(const shd_ctx *ctx, const T *Ip, T *Sp, const T *mom, const T *Sprev,
                                  bool have_prev, int *grid_used, cudaStream_t st);

// Ng acceleration: FP64 inner products of the last four source iterates
// into out5 (part: nblk * 5 doubles of scratch), and the extrapolation
template <class T>
cudaError_t launch_ng_dots(const T *x0, const T *x1, const T *x2, const T *x3, long long n, double *part, int nblk,
                           double *out5, cudaStream_t st);
template <class T>
cudaError_t launch_ng_combine(T *x0, const T *x1, const T *x2, long long n, double a, double b, cudaStream_t st);
// one Runge-Kutta combination pass over a discrete-ordinate array (App. A)
template <class T>
cudaError_t launch_rk_stage(T *I, const T *A, T *B, T *acc, long long n, double cnext, bool first, bool last,
                            cudaStream_t st);

// one thread waits on an mbarrier nothing arrives on, `polls` times at most,
// then raises *flag (the bounded-wait failure path of the tensor-core kernels)
cudaError_t launch_wait_selftest(long long polls, int *flag, cudaStream_t st);

// a2 on the tensor cores for group-mixing kernels (MIXED): usable, its
// operands (built from d_K into d_tcK), and the source + partial sums pass
bool source_tc_usable(const shd_ctx *ctx);
size_t source_tc_operand_bytes(const shd_ctx *ctx);
cudaError_t launch_source_tc_operands(shd_ctx *ctx, cudaStream_t st);
cudaError_t launch_source_sums_tc(shd_ctx *ctx, const float *Ip, float *Sp, const float *mom, const float *Sprev,
                                  bool have_prev, int *grid_used, cudaStream_t st);

size_t remap_smem_bytes(const shd_ctx *ctx);
template <class T>
cudaError_t launch_project_nm(const shd_ctx *ctx, const T *I, T *Ip, T *mom, T *nm0, T *nm1, cudaStream_t st);
size_t sh2lab_tile_smem_bytes(const shd_ctx *ctx);
size_t sweep_smem_bytes(const shd_ctx *ctx);

}  // namespace shd
