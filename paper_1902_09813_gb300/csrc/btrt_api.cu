// btrt_api.cu -- host runtime and C ABI of the B-TriRT D2Q9 solver (see include/btrt.h).
//
// A lattice lives entirely in a caller-owned device workspace:
//   [F buffer 0: 9 planes][F buffer 1: 9 planes][phi plane 0][phi plane 1][trig tables]
//   [wall arrays][reduction scratch][residual partials][optional field planes]
// Planes are row major with a row pitch of nx rounded up to 64 elements; every
// region starts on a 256-byte boundary.  Populations and phi are double
// buffered: a launch reads buffer `cur` and writes buffer 1 - cur (one step per
// launch, or two in the two-step form of FP32 compute).
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/btrt.h"
#include "btrt_internal.h"

#include <cudaTypedefs.h>

using namespace btrt;

namespace {

thread_local std::string g_err;

btrt_status fail(btrt_status code, const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
    return code;
}

#define CUDA_TRY(expr)                                                                    \
    do {                                                                                  \
        cudaError_t e_ = (expr);                                                          \
        if (e_ != cudaSuccess)                                                            \
            return fail(BTRT_ECUDA, "%s: %s (%s:%d)", #expr, cudaGetErrorString(e_),    \
                        __FILE__, __LINE__);                                              \
    } while (0)

constexpr size_t kAlign = 256;

size_t align_up(size_t v, size_t a) { return (v + a - 1) / a * a; }

// cuTensorMapEncodeTiled from the driver, looked up once through the runtime.
PFN_cuTensorMapEncodeTiled_v12000 tensor_map_encoder() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    static bool tried = false;
    if (!tried) {
        tried = true;
        void *ptr = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &ptr, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(ptr);
        else
            cudaGetLastError();
    }
    return fn;
}

// 3-D tensor map over one population buffer: {x: nx, y: ny, plane: 9}.
bool encode_buffer_map(CUtensorMap *map, void *base, const btrt_grid_desc &g, long long pitch, long long plane,
                       int box_x, int box_y) {
    PFN_cuTensorMapEncodeTiled_v12000 enc = tensor_map_encoder();
    if (!enc) return false;
    const size_t es = elem_size(g.storage);
    const CUtensorMapDataType dt = g.storage == BTRT_F32 ? CU_TENSOR_MAP_DATA_TYPE_FLOAT32 : CU_TENSOR_MAP_DATA_TYPE_UINT16;
    const cuuint64_t dims[3] = {(cuuint64_t)g.nx, (cuuint64_t)g.ny, 9};
    const cuuint64_t strides[2] = {(cuuint64_t)(pitch * es), (cuuint64_t)(plane * es)};
    const cuuint32_t box[3] = {(cuuint32_t)box_x, (cuuint32_t)box_y, 9};
    const cuuint32_t estr[3] = {1, 1, 1};
    return enc(map, dt, 3, base, dims, strides, box, estr, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_NONE,
               CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

btrt_status check_desc(const btrt_grid_desc *g) {
    if (!g) return fail(BTRT_EINVAL, "null grid description");
    if (g->nx < 3 || g->ny < 3 || g->nx > 65536 || g->ny > 65536)
        return fail(BTRT_EINVAL, "grid %d x %d outside [3, 65536]", g->nx, g->ny);
    for (int k = 0; k < 4; ++k)
        if (g->bc[k] != BTRT_BC_PERIODIC && g->bc[k] != BTRT_BC_HBB)
            return fail(BTRT_EINVAL, "bc[%d] = %d is not a boundary kind", k, g->bc[k]);
    if (g->bc[0] != g->bc[1] || g->bc[2] != g->bc[3])
        return fail(BTRT_EINVAL, "opposite sides must share the boundary kind");
    if (g->compute == BTRT_F64) {
        if (g->storage != BTRT_F64)
            return fail(BTRT_EINVAL, "FP64 compute requires FP64 storage");
    } else if (g->compute == BTRT_DF64) {
        if (g->storage != BTRT_DF64)
            return fail(BTRT_EINVAL, "double-word compute requires double-word storage");
    } else if (g->compute == BTRT_F32) {
        if (g->storage != BTRT_F32 && g->storage != BTRT_F16 && g->storage != BTRT_BF16)
            return fail(BTRT_EINVAL, "FP32 compute takes F32, F16 or BF16 storage");
    } else {
        return fail(BTRT_EINVAL, "compute must be BTRT_F64, BTRT_DF64 or BTRT_F32");
    }
    if (!(g->dx > 0.0) || !(g->dt > 0.0) || !std::isfinite(g->dx) || !std::isfinite(g->dt))
        return fail(BTRT_EINVAL, "dx and dt must be positive and finite");
    if (!std::isfinite(g->phi_ref) || !std::isfinite(g->x0) || !std::isfinite(g->y0))
        return fail(BTRT_EINVAL, "phi_ref, x0, y0 must be finite");
    if (g->fields & ~(BTRT_FIELD_SOURCE | BTRT_FIELD_DIFFUSION))
        return fail(BTRT_EINVAL, "unknown field bits 0x%x", g->fields);
    if (g->shift < BTRT_SHIFT_REF || g->shift > BTRT_SHIFT_MOMENT_SR)
        return fail(BTRT_EINVAL, "unknown storage shift %d", g->shift);
    if (has_phi_lo(*g) && g->compute != BTRT_F32)
        return fail(BTRT_EINVAL, "the double-word phi planes of BTRT_SHIFT_LOCAL_DW(_SR) serve FP32 compute");
    if (stochastic_store(*g) && (g->compute != BTRT_F32 || (g->storage != BTRT_F16 && g->storage != BTRT_BF16)))
        return fail(BTRT_EINVAL, "stochastic rounding (BTRT_SHIFT_LOCAL_SR, _DW_SR, _MOMENT_SR) serves F16/BF16 storage "
                    "with FP32 compute");
    const long long pitch = (long long)((g->nx + 63) / 64) * 64;
    if (9 * pitch * (long long)g->ny >= (1LL << 31))
        return fail(BTRT_EINVAL, "grid %d x %d: the nine padded planes must hold fewer than 2^31 values "
                    "(about 238 M nodes)", g->nx, g->ny);
    return BTRT_OK;
}

Layout make_layout(const btrt_grid_desc *g) {
    Layout L;
    const size_t sf = elem_size(g->storage);
    const size_t sr = elem_size(g->compute);
    L.pitch = (long long)align_up((size_t)g->nx, 64);
    L.plane = L.pitch * (long long)g->ny;
    L.maxside = g->nx > g->ny ? g->nx : g->ny;
    L.fbuf_bytes = align_up(9 * (size_t)L.plane * sf, kAlign);
    size_t off = 0;
    L.off_f[0] = off;
    off += L.fbuf_bytes;
    L.off_f[1] = off;
    off += L.fbuf_bytes;
    // a double-word phi (BTRT_SHIFT_LOCAL_DW, _DW_SR) keeps its low words in a second plane
    const size_t phi_planes = has_phi_lo(*g) ? 2 : 1;
    // BTRT_SHIFT_MOMENT_SR keeps the writers' first moments in two planes of the
    // storage format after the phi plane
    const size_t j_bytes = has_j(*g) ? 2 * (size_t)L.plane * sf : 0;
    for (int k = 0; k < 2; ++k) {
        L.off_phi[k] = off;
        off += align_up(phi_planes * (size_t)L.plane * sr + j_bytes, kAlign);
    }
    L.off_tab = off;
    off += align_up(2 * ((size_t)g->nx + (size_t)g->ny) * sr, kAlign);
    L.off_wall = off;
    off += align_up(4 * (size_t)L.maxside * sr, kAlign);
    L.off_red = off;
    off += align_up((kRedBlocks + 2) * sizeof(double) + 16, kAlign);
    L.resid_blocks = sweep_blocks(g->nx, g->ny, g->compute, g->storage);
    L.off_resid = off;
    off += align_up((size_t)L.resid_blocks * sizeof(double), kAlign);
    if (g->fields & BTRT_FIELD_SOURCE) {
        L.off_srcf = off;
        off += align_up((size_t)L.plane * sr, kAlign);
    }
    if (g->fields & BTRT_FIELD_DIFFUSION) {
        L.off_af = off;
        off += align_up(3 * (size_t)L.plane * sr, kAlign);
    }
    L.total = off;
    return L;
}

// ---------------------------------------------------------------- small kernels
template <typename Real, typename In>
__global__ void dense_to_plane(const In *__restrict__ src, Real *__restrict__ dst, int nx, int ny,
                               long long pitch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x < nx && y < ny) dst[(long long)y * pitch + x] = Real((double)src[(long long)y * nx + x]);
}

// Low words of a double-word phi plane: v - (float)v, rounded to FP32.
template <typename In>
__global__ void dense_to_plane_lo(const In *__restrict__ src, float *__restrict__ lo, int nx, int ny,
                                  long long pitch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x < nx && y < ny) {
        const double v = (double)src[(long long)y * nx + x];
        lo[(long long)y * pitch + x] = (float)(v - (double)(float)v);
    }
}

// A double-word phi plane (high and low words) as dense FP64 or FP32 values.
template <typename Out>
__global__ void dw_planes_to_dense(const float *__restrict__ hi, const float *__restrict__ lo, Out *__restrict__ dst,
                                   int nx, int ny, long long pitch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x < nx && y < ny)
        dst[(long long)y * nx + x] = (Out)((double)hi[(long long)y * pitch + x] + (double)lo[(long long)y * pitch + x]);
}

template <typename Real, typename Out>
__global__ void plane_to_dense(const Real *__restrict__ src, Out *__restrict__ dst, int nx, int ny,
                               long long pitch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    const int y = blockIdx.y;
    if (x < nx && y < ny) dst[(long long)y * nx + x] = (Out) static_cast<double>(src[(long long)y * pitch + x]);
}

}  // namespace

void btrt::set_last_error(const char *fmt, ...) {
    char buf[512];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof buf, fmt, ap);
    va_end(ap);
    g_err = buf;
}

double btrt::half_bits_to_double(int fmt, const unsigned char *p) {
    uint16_t b;
    std::memcpy(&b, p, 2);
    if (fmt == BTRT_BF16) {
        uint32_t u = (uint32_t)b << 16;
        float f;
        std::memcpy(&f, &u, 4);
        return f;
    }
    // IEEE binary16 -> double, by its definition
    const int sign = (b >> 15) & 1, e = (b >> 10) & 31, m = b & 1023;
    double v;
    if (e == 0) v = std::ldexp((double)m, -24);
    else if (e == 31) v = m ? NAN : INFINITY;
    else v = std::ldexp((double)(m | 1024), e - 25);
    return sign ? -v : v;
}

size_t btrt::elem_size(int fmt) {
    switch (fmt) {
    case BTRT_F64: return 8;
    case BTRT_F32: return 4;
    case BTRT_F16: return 2;
    case BTRT_BF16: return 2;
    case BTRT_DF64: return 8;
    default: return 0;
    }
}

void btrt::step_scalars(btrt_lattice L, int64_t n, bool first, double *src_val, double *wall_fac) {
    const btrt_grid_desc &g = L->g;
    const btrt_coeffs &c = L->c;
    const double tn = L->t0 + (double)n * g.dt;
    // bounce-back values of the streaming that ends at t_n
    *wall_fac = c.wall_lam == 0.0 ? 1.0 : std::exp(c.wall_lam * tn);
    if (c.src_kind == BTRT_SRC_CONST) {
        *src_val = c.src_const * g.dt;
    } else if (c.src_kind == BTRT_SRC_REACTION) {
        *src_val = g.dt;   // times (3 S(phi^n) - S(phi^{n-1})) / 2, evaluated per node
    } else if (c.src_kind == BTRT_SRC_TRIG || c.src_kind == BTRT_SRC_FIELD) {
        // dt S_i + dt^2/2 (S_i^n - S_i^{n-1})/dt = w_i dt (3 S^n - S^{n-1}) / 2 (scheme 2)
        const double Tn = std::exp(c.src_lam * tn);
        const double Tp = first ? Tn : std::exp(c.src_lam * (tn - g.dt));
        *src_val = g.dt * 0.5 * (3.0 * Tn - Tp);
    } else {
        *src_val = 0.0;
    }
}

template <typename Real>
void btrt::fill_params(btrt_lattice L, SweepParams<Real> &p, int64_t n, bool first) {
    const btrt_grid_desc &g = L->g;
    const btrt_coeffs &c = L->c;
    std::memset(&p, 0, sizeof p);
    // the initialising collision rewrites the current buffers in place (no streaming)
    p.fin = L->fbuf(L->cur);
    p.fout = L->fbuf(first ? L->cur : 1 - L->cur);
    p.phi_in = L->phi<Real>(L->cur);
    p.phi_out = L->phi<Real>(first ? L->cur : 1 - L->cur);
    if constexpr (std::is_same<Real, float>::value) {
        p.phi_in_lo = L->phi_lo(L->cur);
        p.phi_out_lo = L->phi_lo(first ? L->cur : 1 - L->cur);
        p.j_in = L->jplanes(L->cur);
        p.j_out = L->jplanes(first ? L->cur : 1 - L->cur);
    }
    p.nx = g.nx;
    p.ny = g.ny;
    p.pitch = (int)L->lay.pitch;
    p.plane = (int)L->lay.plane;
    p.hbb_x = g.bc[0] == BTRT_BC_HBB;
    p.hbb_y = g.bc[2] == BTRT_BC_HBB;
    const double w[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    for (int i = 0; i < 9; ++i) p.wref[i] = shift_of(g) == kShiftRef ? (Real)(w[i] * g.phi_ref) : (Real)0.0;
    for (int s = 0; s < 4; ++s) {
        p.wall_const[s] = (Real)L->wall_const[s];
        p.wall_arr[s] = L->wall_is_arr[s] ? L->wall<Real>(s) : nullptr;
    }
    double src_val = 0.0, wall_fac = 1.0;
    step_scalars(L, n, first, &src_val, &wall_fac);
    p.wall_fac = (Real)wall_fac;
    p.ux = (Real)L->ux;
    p.uy = (Real)L->uy;
    p.b2 = (Real)L->b2;
    p.bgx = (Real)L->bgx;
    p.bgy = (Real)L->bgy;
    p.bq = (Real)L->bq;
    p.bq2 = L->bq == 2.0 ? 1 : 0;
    p.react_rate = (Real)c.react_rate;
    p.react_exp = (Real)c.react_exp;
    p.react2 = c.react_exp == 2.0 ? 1 : 0;
    half_split(L->bq, &p.bq_n, &p.bq_h);
    half_split(c.react_exp, &p.re_n, &p.re_h);
    p.c3 = (Real)c.c3;
    p.A0xx = (Real)L->A0[0];
    p.A0xy = (Real)L->A0[1];
    p.A0yy = (Real)L->A0[2];
    p.a2 = (Real)c.a2;
    p.k0 = (Real)c.k0;
    p.nonlin_A = L->nonlin_A ? 1 : 0;
    p.k2_hbb = c.k2_mode == BTRT_K2_HBB;
    p.k2c = (Real)c.k2;
    p.K1xx = (Real)L->K1[0];
    p.K1xy = (Real)L->K1[1];
    p.K1yy = (Real)L->K1[2];
    p.k2 = (Real)L->k2;
    p.cond_limit = (Real)1.0e4;
    for (int k = 0; k < 3; ++k) p.A0d[k] = L->A0[k];
    p.a2d = c.a2;
    p.src_kind = c.src_kind;
    p.src_val = (Real)src_val;
    p.srcF = L->srcf<Real>();
    p.Af = L->have_af ? L->af<Real>() : nullptr;
    if (c.src_kind == BTRT_SRC_TRIG) {
        Real *tb = L->tab<Real>();
        p.Xs = tb;
        p.Xc = tb + g.nx;
        p.Ys = tb + 2 * g.nx;
        p.Yc = tb + 2 * g.nx + g.ny;
    }
    p.k0_one = c.k0 == 1.0 ? 1 : 0;
    p.first = first ? 1 : 0;
    p.flags = L->flags();
    // constants of the folded collision
    {
        const double k0 = c.k0, K1xx = L->K1[0], K1xy = L->K1[1], K1yy = L->K1[2];
        const double dk = L->k2 - k0;
        const double Px = K1xx * L->ux + K1xy * L->uy, Py = K1xy * L->ux + K1yy * L->uy;
        const double gx = L->ux - 0.5 * Px, gy = L->uy - 0.5 * Py;
        FoldConsts<Real> &q = p.lin;
        q.Px = (Real)Px;
        q.Py = (Real)Py;
        q.Qxx = (Real)(K1xx - k0);
        q.Qxy = (Real)K1xy;
        q.Qyy = (Real)(K1yy - k0);
        q.gx = (Real)gx;
        q.gy = (Real)gy;
        q.Pgx = (Real)(Px + gx);
        q.Pgy = (Real)(Py + gy);
        q.k0 = (Real)k0;
        q.om = (Real)(1.0 - k0);
        q.k0x15 = (Real)(1.5 * k0);
        q.c0 = (Real)(2.0 * dk / 3.0);
        q.k6 = (Real)(-dk / 12.0);
        q.k6x3 = (Real)(-dk / 4.0);
        q.c0k = (Real)(-2.0 * k0 / 3.0);
        q.k6k = (Real)(k0 / 12.0);
        q.k6x3k = (Real)(k0 / 4.0);
        q.a2x3 = (Real)(3.0 * c.a2);
    }
    // the reference value of kShiftRef storage (zero otherwise)
    p.phi_ref = shift_of(g) == kShiftRef ? (Real)g.phi_ref : (Real)0.0;
    // stochastic rounding: the seed of step index n (the same in every kernel form)
    p.sr_seed = sr_step_seed(n);
}

template void btrt::fill_params<double>(btrt_lattice, SweepParams<double> &, int64_t, bool);
template void btrt::fill_params<float>(btrt_lattice, SweepParams<float> &, int64_t, bool);
template void btrt::fill_params<dw>(btrt_lattice, SweepParams<dw> &, int64_t, bool);

// Which compiled variant of the sweep serves these coefficients.
int btrt::sweep_mode(btrt_lattice L) {
    const btrt_coeffs &c = L->c;
    const bool linear = c.b2 == 0.0 && c.c3 == 0.0 && c.a2 == 0.0 && !L->have_af;
    if (!linear) return kGeneral;
    if (L->g.compute == BTRT_F64 && c.k0 == 1.0) return kLinearK0One;
    return kLinear;
}

// The kernel form BTRT_SWEEP_AUTO stands for, as measured on GB300 at 8192^2: the
// one-step vector form for FP16/BF16 storage (manufactured solution 140-153
// GLUPS against 119-141 for the two-step forms; nonlinear workload 117-130
// against 77-116), the scalar two-step form for FP32 storage (116-124 and
// 103-114 GLUPS against 110-117 and 69-79 with vector access, 80-86 for one step
// per launch).  Lattices below kVecAutoNodes nodes take the two-step form with
// every storage: a step there lasts a few microseconds, launches dominate, and
// two steps per launch halve them (512 instances of 32^2 to 1024^2 nodes, 2000
// steps each, one after the other: 10.5 s with the vector form, 6.8 s with two
// steps per launch).
// Stochastically rounded storage has the plain and vector forms only: the vector
// form from kVecAutoNodes on, the plain one below.
constexpr long long kVecAutoNodes = 1LL << 21;
int btrt::effective_sweep_variant(btrt_lattice L) {
    if (L->g.compute != BTRT_F32 || has_phi_lo(L->g)) return BTRT_SWEEP_PLAIN;
    if (L->sweep_variant != BTRT_SWEEP_AUTO) return L->sweep_variant;
    const bool s16 = L->g.storage == BTRT_F16 || L->g.storage == BTRT_BF16;
    const bool large = (long long)L->g.nx * L->g.ny >= kVecAutoNodes;
    if (stochastic_store(L->g)) return large ? BTRT_SWEEP_VEC : BTRT_SWEEP_PLAIN;
    return s16 && large ? BTRT_SWEEP_VEC : BTRT_SWEEP_TB2;
}

namespace {

btrt_status launch(btrt_lattice L, int64_t n, bool first, bool resid = false) {
    if (L->g.compute == BTRT_F64) {
        SweepParams<double> p;
        fill_params(L, p, n, first);
        if (resid) p.resid_partials = L->resid_partials();
        CUDA_TRY(launch_sweep_f64(p, sweep_mode(L), L->stream));
    } else if (L->g.compute == BTRT_DF64) {
        SweepParams<dw> p;
        fill_params(L, p, n, first);
        if (resid) p.resid_partials = L->resid_partials();
        CUDA_TRY(launch_sweep_dw(p, sweep_mode(L), L->stream));
    } else {
        SweepParams<float> p;
        fill_params(L, p, n, first);
        if (resid) p.resid_partials = L->resid_partials();
        const int sh = shift_of(L->g);
        if (!first && !resid && L->have_tma && L->sweep_variant == BTRT_SWEEP_TMA)
            CUDA_TRY(launch_sweep_tma(p, L->g.storage, sh, sweep_mode(L), &L->tma_in[L->cur],
                                      &L->tma_out[1 - L->cur], L->stream));
        else if (!first && !resid && effective_sweep_variant(L) == BTRT_SWEEP_VEC)
            CUDA_TRY(launch_sweep_vec(p, L->g.storage, sh, sweep_mode(L), L->stream));
        else
            CUDA_TRY(launch_sweep_f32(p, L->g.storage, sh, sweep_mode(L), L->stream));
    }
    return BTRT_OK;
}

// Dense host arrays (row major, nx*ny) -> pitched device planes of Real, scaled.
template <typename Real>
btrt_status upload_planes(btrt_lattice L, Real *dst, const double *const *src, int nplanes, double scale) {
    const btrt_grid_desc &g = L->g;
    std::vector<Real> h((size_t)nplanes * L->lay.plane, Real(0.0));
    for (int k = 0; k < nplanes; ++k)
        for (int y = 0; y < g.ny; ++y)
            for (int x = 0; x < g.nx; ++x)
                h[(size_t)k * L->lay.plane + (size_t)y * L->lay.pitch + x] =
                    Real(scale * src[k][(size_t)y * g.nx + x]);
    CUDA_TRY(cudaMemcpyAsync(dst, h.data(), h.size() * sizeof(Real), cudaMemcpyHostToDevice, L->stream));
    CUDA_TRY(cudaStreamSynchronize(L->stream));
    return BTRT_OK;
}

template <typename Real>
btrt_status upload_tables(btrt_lattice L) {
    const btrt_grid_desc &g = L->g;
    const btrt_coeffs &c = L->c;
    std::vector<Real> h(2 * ((size_t)g.nx + g.ny));
    for (int i = 0; i < g.nx; ++i) {
        const double x = g.x0 + (i + 0.5) * g.dx;
        h[i] = (Real)std::sin(c.src_k * x);
        h[g.nx + i] = (Real)std::cos(c.src_k * x);
    }
    for (int j = 0; j < g.ny; ++j) {
        const double y = g.y0 + (j + 0.5) * g.dx;
        const double sy = std::sin(c.src_k * y), cy = std::cos(c.src_k * y);
        // alpha folded in: S_spatial = Xs (a_ss sy + a_sc cy) + Xc (a_cs sy + a_cc cy)
        h[2 * g.nx + j] = (Real)(c.src_alpha[0] * sy + c.src_alpha[1] * cy);
        h[2 * g.nx + g.ny + j] = (Real)(c.src_alpha[2] * sy + c.src_alpha[3] * cy);
    }
    CUDA_TRY(cudaMemcpyAsync(L->tab<Real>(), h.data(), h.size() * sizeof(Real),
                             cudaMemcpyHostToDevice, L->stream));
    CUDA_TRY(cudaStreamSynchronize(L->stream));
    return BTRT_OK;
}

template <typename Real>
btrt_status upload_wall(btrt_lattice L, int side, const double *v, int n) {
    std::vector<Real> h(n);
    for (int k = 0; k < n; ++k) h[k] = (Real)v[k];
    CUDA_TRY(cudaMemcpyAsync(L->wall<Real>(side), h.data(), n * sizeof(Real),
                             cudaMemcpyHostToDevice, L->stream));
    CUDA_TRY(cudaStreamSynchronize(L->stream));
    return BTRT_OK;
}

// phi0 -> phi plane 0 (the initialising collision then runs with cur = 0).
template <typename Real>
btrt_status stage_phi0(btrt_lattice L, const void *phi0, int dtype, int on_device) {
    const btrt_grid_desc &g = L->g;
    const size_t n = (size_t)g.nx * g.ny;
    const size_t bytes = n * elem_size(dtype);
    const void *dev_src = phi0;
    if (!on_device) {
        // stage the dense host array in population buffer 1 (overwritten below)
        if (bytes > L->lay.fbuf_bytes) return fail(BTRT_ENOMEM, "staging area too small");
        CUDA_TRY(cudaMemcpyAsync(L->fbuf(1), phi0, bytes, cudaMemcpyHostToDevice, L->stream));
        dev_src = L->fbuf(1);
    }
    const dim3 blk(256), grd((unsigned)((g.nx + 255) / 256), (unsigned)g.ny);
    if (dtype == BTRT_F64)
        dense_to_plane<Real, double><<<grd, blk, 0, L->stream>>>((const double *)dev_src, L->phi<Real>(0),
                                                                 g.nx, g.ny, L->lay.pitch);
    else
        dense_to_plane<Real, float><<<grd, blk, 0, L->stream>>>((const float *)dev_src, L->phi<Real>(0),
                                                                g.nx, g.ny, L->lay.pitch);
    CUDA_TRY(cudaGetLastError());
    if (L->phi_lo(0)) {
        if (dtype == BTRT_F64)
            dense_to_plane_lo<double><<<grd, blk, 0, L->stream>>>((const double *)dev_src, L->phi_lo(0), g.nx, g.ny,
                                                                 L->lay.pitch);
        else
            dense_to_plane_lo<float><<<grd, blk, 0, L->stream>>>((const float *)dev_src, L->phi_lo(0), g.nx, g.ny,
                                                                L->lay.pitch);
        CUDA_TRY(cudaGetLastError());
    }
    if (!on_device) CUDA_TRY(cudaStreamSynchronize(L->stream));  // host buffer may be reused
    return BTRT_OK;
}

template <typename Real>
btrt_status copy_phi_out(btrt_lattice L, void *dst, int dtype, int on_device) {
    const btrt_grid_desc &g = L->g;
    const size_t n = (size_t)g.nx * g.ny;
    if (L->phi_lo(L->cur)) {
        // double-word phi: high + low word, in FP64 (or rounded once to FP32)
        const dim3 blk(256), grd((unsigned)((g.nx + 255) / 256), (unsigned)g.ny);
        void *out = dst;
        if (!on_device) {
            if (n * elem_size(dtype) > L->lay.fbuf_bytes) return fail(BTRT_ENOMEM, "staging area too small");
            out = L->fbuf(1 - L->cur);   // the other population buffer: rewritten by the next step anyway
        }
        if (dtype == BTRT_F64)
            dw_planes_to_dense<double><<<grd, blk, 0, L->stream>>>(L->phi<float>(L->cur), L->phi_lo(L->cur),
                                                                   (double *)out, g.nx, g.ny, L->lay.pitch);
        else
            dw_planes_to_dense<float><<<grd, blk, 0, L->stream>>>(L->phi<float>(L->cur), L->phi_lo(L->cur),
                                                                  (float *)out, g.nx, g.ny, L->lay.pitch);
        CUDA_TRY(cudaGetLastError());
        if (!on_device) {
            CUDA_TRY(cudaMemcpyAsync(dst, out, n * elem_size(dtype), cudaMemcpyDeviceToHost, L->stream));
            CUDA_TRY(cudaStreamSynchronize(L->stream));
        }
        return BTRT_OK;
    }
    if (on_device) {
        const dim3 blk(256), grd((unsigned)((g.nx + 255) / 256), (unsigned)g.ny);
        if (dtype == BTRT_F64)
            plane_to_dense<Real, double><<<grd, blk, 0, L->stream>>>(L->phi<Real>(), (double *)dst,
                                                                     g.nx, g.ny, L->lay.pitch);
        else
            plane_to_dense<Real, float><<<grd, blk, 0, L->stream>>>(L->phi<Real>(), (float *)dst,
                                                                    g.nx, g.ny, L->lay.pitch);
        CUDA_TRY(cudaGetLastError());
        return BTRT_OK;
    }
    if (L->g.compute != BTRT_DF64 && dtype == (sizeof(Real) == 8 ? BTRT_F64 : BTRT_F32)) {
        CUDA_TRY(cudaMemcpy2DAsync(dst, g.nx * sizeof(Real), L->phi<Real>(), L->lay.pitch * sizeof(Real),
                                   g.nx * sizeof(Real), g.ny, cudaMemcpyDeviceToHost, L->stream));
        CUDA_TRY(cudaStreamSynchronize(L->stream));
        return BTRT_OK;
    }
    std::vector<Real> h(n);
    CUDA_TRY(cudaMemcpy2DAsync(h.data(), g.nx * sizeof(Real), L->phi<Real>(), L->lay.pitch * sizeof(Real),
                               g.nx * sizeof(Real), g.ny, cudaMemcpyDeviceToHost, L->stream));
    CUDA_TRY(cudaStreamSynchronize(L->stream));
    if (dtype == BTRT_F64)
        for (size_t k = 0; k < n; ++k) ((double *)dst)[k] = static_cast<double>(h[k]);
    else
        for (size_t k = 0; k < n; ++k) ((float *)dst)[k] = (float)static_cast<double>(h[k]);
    return BTRT_OK;
}

template <typename Real>
btrt_status reduce_phi(btrt_lattice L, double *out) {
    const btrt_grid_desc &g = L->g;
    CUDA_TRY(enqueue_rows_sum<Real>(L->phi<Real>(), g.nx, g.ny, L->lay.pitch, L->partials(), L->red_out(),
                                    L->stream));
    CUDA_TRY(cudaMemcpyAsync(out, L->red_out(), sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CUDA_TRY(cudaStreamSynchronize(L->stream));
    if (L->phi_lo(L->cur)) {
        // double-word phi: the low words' sum, same fixed order, added once
        double lo = 0.0;
        CUDA_TRY(enqueue_rows_sum<float>(L->phi_lo(L->cur), g.nx, g.ny, L->lay.pitch, L->partials(), L->red_out(),
                                         L->stream));
        CUDA_TRY(cudaMemcpyAsync(&lo, L->red_out(), sizeof(double), cudaMemcpyDeviceToHost, L->stream));
        CUDA_TRY(cudaStreamSynchronize(L->stream));
        *out += lo;
    }
    return BTRT_OK;
}


struct StateHeader {
    char magic[8];
    int32_t nx, ny, compute, storage;
    int64_t step;
    double t0;
    int32_t shift, pad;   // storage shift of the saved populations
};

}  // namespace

// ---------------------------------------------------------------- C ABI
extern "C" {

size_t btrt_workspace_bytes(const btrt_grid_desc *g) {
    if (check_desc(g) != BTRT_OK) return 0;
    return make_layout(g).total;
}

btrt_status btrt_create(const btrt_grid_desc *g, void *dev_workspace, size_t workspace_bytes,
                        void *cuda_stream, btrt_lattice *out) {
    if (!out) return fail(BTRT_EINVAL, "null output handle");
    *out = nullptr;
    btrt_status st = check_desc(g);
    if (st != BTRT_OK) return st;
    if (!dev_workspace) return fail(BTRT_EINVAL, "null workspace");
    if (((uintptr_t)dev_workspace) % kAlign) return fail(BTRT_EINVAL, "workspace not 256-byte aligned");
    Layout lay = make_layout(g);
    if (workspace_bytes < lay.total)
        return fail(BTRT_ENOMEM, "workspace of %zu bytes < required %zu", workspace_bytes, lay.total);
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, dev_workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail(BTRT_EINVAL, "workspace is not device memory");
    }
    btrt_lattice L = new (std::nothrow) btrt_lattice_s();
    if (!L) return fail(BTRT_ENOMEM, "host allocation failed");
    L->g = *g;
    L->lay = lay;
    L->ws = static_cast<unsigned char *>(dev_workspace);
    L->stream = static_cast<cudaStream_t>(cuda_stream);
    std::memset(&L->c, 0, sizeof L->c);
    L->c.k0 = 1.0;
    cudaError_t e = cudaMemsetAsync(L->flags(), 0, 16, L->stream);
    if (e != cudaSuccess) {
        delete L;
        return fail(BTRT_ECUDA, "cudaMemsetAsync: %s", cudaGetErrorString(e));
    }
    if (g->compute == BTRT_F32 && !has_phi_lo(*g) && !stochastic_store(*g)) {
        int bix, biy, box, boy;
        tma_box(g->storage, &bix, &biy, &box, &boy);
        bool ok = true;
        for (int k = 0; k < 2; ++k) {
            ok = ok && encode_buffer_map(&L->tma_in[k], L->fbuf(k), *g, lay.pitch, lay.plane, bix, biy);
            ok = ok && encode_buffer_map(&L->tma_out[k], L->fbuf(k), *g, lay.pitch, lay.plane, box, boy);
        }
        L->have_tma = ok;
    }
    *out = L;
    return BTRT_OK;
}

btrt_status btrt_set_coeffs(btrt_lattice L, const btrt_coeffs *c) {
    if (!L || !c) return fail(BTRT_EINVAL, "null argument");
    const btrt_grid_desc &g = L->g;
    const double cl = g.dx / g.dt;                 // lattice speed c
    const double axx = c->A0[0], axy = c->A0[1], ayy = c->A0[2];
    if (!(axx > 0.0) || !(ayy > 0.0) || !(axx * ayy - axy * axy > 0.0))
        return fail(BTRT_EINVAL, "A0 must be symmetric positive definite");
    if (!(c->k0 > 0.0 && c->k0 < 2.0)) return fail(BTRT_EINVAL, "k0 = %g outside (0, 2)", c->k0);
    if (c->k2_mode != BTRT_K2_HBB && c->k2_mode != BTRT_K2_CONST)
        return fail(BTRT_EINVAL, "unknown k2 mode %d", c->k2_mode);
    if (c->k2_mode == BTRT_K2_CONST && !(c->k2 > 0.0 && c->k2 < 2.0))
        return fail(BTRT_EINVAL, "k2 = %g outside (0, 2)", c->k2);
    if (c->src_kind < BTRT_SRC_NONE || c->src_kind > BTRT_SRC_REACTION)
        return fail(BTRT_EINVAL, "unknown source kind %d", c->src_kind);
    if (c->src_kind == BTRT_SRC_REACTION && (!std::isfinite(c->react_rate) || !(c->react_exp > 0.0)))
        return fail(BTRT_EINVAL, "reaction source needs a finite rate and an exponent > 0");
    if (!(c->b_q == 0.0 || (c->b_q >= 1.0 && std::isfinite(c->b_q))))
        return fail(BTRT_EINVAL, "flux exponent b_q = %g: must be 0 (default 2) or >= 1", c->b_q);
    if (!std::isfinite(c->b_dir[0]) || !std::isfinite(c->b_dir[1]))
        return fail(BTRT_EINVAL, "non-finite flux direction");
    if (c->src_kind == BTRT_SRC_FIELD && !(g.fields & BTRT_FIELD_SOURCE))
        return fail(BTRT_EINVAL, "BTRT_SRC_FIELD needs BTRT_FIELD_SOURCE in the grid description");
    if (!std::isfinite(c->a2) || c->a2 < 0.0) return fail(BTRT_EINVAL, "a2 must be >= 0");
    L->c = *c;
    // lattice units: B^ = B dt/dx, A^ = A dt/dx^2
    L->ux = c->u[0] / cl;
    L->uy = c->u[1] / cl;
    L->b2 = c->b2 / cl;
    // power-law flux b2 (phi^q / q) d -> bg phi^q in lattice units
    const double q = c->b_q == 0.0 ? 2.0 : c->b_q;
    const bool dflt = c->b_dir[0] == 0.0 && c->b_dir[1] == 0.0;
    L->bq = q;
    L->bgx = L->b2 * (dflt ? 1.0 : c->b_dir[0]) / q;
    L->bgy = L->b2 * (dflt ? 1.0 : c->b_dir[1]) / q;
    const double sA = g.dt / (g.dx * g.dx);
    L->A0[0] = axx * sA;
    L->A0[1] = axy * sA;
    L->A0[2] = ayy * sA;
    // K1 = (3 A^ + I/2)^{-1} at A = A0 (Eq. 30), k2 from Eq. 62 or constant
    const double mxx = 3 * L->A0[0] + 0.5, mxy = 3 * L->A0[1], myy = 3 * L->A0[2] + 0.5;
    const double det = mxx * myy - mxy * mxy;
    L->K1[0] = myy / det;
    L->K1[1] = -mxy / det;
    L->K1[2] = mxx / det;
    const double k1eff = 2.0 / (mxx + myy);
    L->k2 = c->k2_mode == BTRT_K2_HBB ? 8.0 * (k1eff - 2.0) / (3.0 * (k1eff - 4.0)) : c->k2;
    L->nonlin_A = c->a2 != 0.0;
    L->have_coeffs = true;
    if (c->src_kind == BTRT_SRC_TRIG) {
        btrt_status st = g.compute == BTRT_F64    ? upload_tables<double>(L)
                         : g.compute == BTRT_DF64 ? upload_tables<dw>(L)
                                                  : upload_tables<float>(L);
        if (st != BTRT_OK) return st;
    }
    return BTRT_OK;
}

btrt_status btrt_set_boundary(btrt_lattice L, int32_t side, const double *phi_w_host, int32_t n) {
    if (!L || !phi_w_host) return fail(BTRT_EINVAL, "null argument");
    if (side < 0 || side > 3) return fail(BTRT_EINVAL, "side %d outside 0..3", side);
    const int len = side < 2 ? L->g.ny : L->g.nx;
    if (n == 1) {
        if (!std::isfinite(phi_w_host[0])) return fail(BTRT_EINVAL, "non-finite wall value");
        L->wall_const[side] = phi_w_host[0];
        L->wall_is_arr[side] = false;
        return BTRT_OK;
    }
    if (n != len) return fail(BTRT_EINVAL, "side %d takes 1 or %d values, got %d", side, len, n);
    for (int k = 0; k < n; ++k)
        if (!std::isfinite(phi_w_host[k])) return fail(BTRT_EINVAL, "non-finite wall value at %d", k);
    btrt_status st = L->g.compute == BTRT_F64    ? upload_wall<double>(L, side, phi_w_host, n)
                     : L->g.compute == BTRT_DF64 ? upload_wall<dw>(L, side, phi_w_host, n)
                                                 : upload_wall<float>(L, side, phi_w_host, n);
    if (st != BTRT_OK) return st;
    L->wall_is_arr[side] = true;
    return BTRT_OK;
}

btrt_status btrt_set_source_field(btrt_lattice L, const double *F_host) {
    if (!L || !F_host) return fail(BTRT_EINVAL, "null argument");
    if (!(L->g.fields & BTRT_FIELD_SOURCE)) return fail(BTRT_EINVAL, "lattice has no source-field plane");
    const size_t n = (size_t)L->g.nx * L->g.ny;
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(F_host[k])) return fail(BTRT_EINVAL, "non-finite source value at %zu", k);
    btrt_status st = L->g.compute == BTRT_F64    ? upload_planes<double>(L, L->srcf<double>(), &F_host, 1, 1.0)
                     : L->g.compute == BTRT_DF64 ? upload_planes<dw>(L, L->srcf<dw>(), &F_host, 1, 1.0)
                                                 : upload_planes<float>(L, L->srcf<float>(), &F_host, 1, 1.0);
    if (st != BTRT_OK) return st;
    L->have_srcf = true;
    return BTRT_OK;
}

btrt_status btrt_set_diffusion_field(btrt_lattice L, const double *Axx, const double *Axy, const double *Ayy) {
    if (!L || !Axx || !Axy || !Ayy) return fail(BTRT_EINVAL, "null argument");
    if (!(L->g.fields & BTRT_FIELD_DIFFUSION)) return fail(BTRT_EINVAL, "lattice has no diffusion-field planes");
    const size_t n = (size_t)L->g.nx * L->g.ny;
    for (size_t k = 0; k < n; ++k)
        if (!(Axx[k] > 0.0) || !(Ayy[k] > 0.0) || !(Axx[k] * Ayy[k] - Axy[k] * Axy[k] > 0.0))
            return fail(BTRT_EINVAL, "diffusion tensor at node %zu is not symmetric positive definite", k);
    // lattice units: A^ = A dt / dx^2
    const double sA = L->g.dt / (L->g.dx * L->g.dx);
    const double *src[3] = {Axx, Axy, Ayy};
    btrt_status st = L->g.compute == BTRT_F64    ? upload_planes<double>(L, L->af<double>(), src, 3, sA)
                     : L->g.compute == BTRT_DF64 ? upload_planes<dw>(L, L->af<dw>(), src, 3, sA)
                                                 : upload_planes<float>(L, L->af<float>(), src, 3, sA);
    if (st != BTRT_OK) return st;
    L->have_af = true;
    return BTRT_OK;
}

btrt_status btrt_init_phi(btrt_lattice L, const void *phi0, int32_t dtype, int32_t on_device, double t0) {
    NvtxRange range("btrt_init_phi");
    if (!L || !phi0) return fail(BTRT_EINVAL, "null argument");
    if (!L->have_coeffs) return fail(BTRT_ESTATE, "btrt_set_coeffs must come before btrt_init_phi");
    if (L->c.src_kind == BTRT_SRC_FIELD && !L->have_srcf)
        return fail(BTRT_ESTATE, "btrt_set_source_field must come before btrt_init_phi");
    if (dtype != BTRT_F64 && dtype != BTRT_F32) return fail(BTRT_EINVAL, "phi0 dtype must be F64 or F32");
    if (!std::isfinite(t0)) return fail(BTRT_EINVAL, "t0 must be finite");
    btrt_status st = L->g.compute == BTRT_F64    ? stage_phi0<double>(L, phi0, dtype, on_device)
                     : L->g.compute == BTRT_DF64 ? stage_phi0<dw>(L, phi0, dtype, on_device)
                                                 : stage_phi0<float>(L, phi0, dtype, on_device);
    if (st != BTRT_OK) return st;
    L->t0 = t0;
    L->step = 0;
    L->cur = 0;
    CUDA_TRY(cudaMemsetAsync(L->flags(), 0, 16, L->stream));
    st = launch(L, 0, true);
    if (st != BTRT_OK) return st;
    L->ready = true;
    return BTRT_OK;
}

btrt_status btrt_step(btrt_lattice L, int64_t nsteps) {
    NvtxRange range("btrt_step");
    if (!L) return fail(BTRT_EINVAL, "null lattice");
    if (!L->ready) return fail(BTRT_ESTATE, "lattice not initialised");
    if (nsteps < 0) return fail(BTRT_EINVAL, "negative step count");
    // the two-step forms serve every FP32-compute lattice (AUTO: see effective_sweep_variant)
    const int form = effective_sweep_variant(L);
    if (form == BTRT_SWEEP_TB2 || form == BTRT_SWEEP_TB2V) {
        // pairs of steps in one launch: inputs from buffer cur, outputs to the other
        for (; nsteps >= 2; nsteps -= 2) {
            SweepParams<float> pa, pb;
            fill_params(L, pa, L->step + 1, false);
            fill_params(L, pb, L->step + 2, false);
            if (form == BTRT_SWEEP_TB2V)
                CUDA_TRY(launch_sweep_tb2v(pa, pb, L->g.storage, shift_of(L->g), sweep_mode(L), L->stream));
            else
                CUDA_TRY(launch_sweep_tb2(pa, pb, L->g.storage, shift_of(L->g), sweep_mode(L), L->stream));
            L->cur = 1 - L->cur;
            L->step += 2;
        }
    }
    for (int64_t k = 0; k < nsteps; ++k) {
        btrt_status st = launch(L, L->step + 1, false);
        if (st != BTRT_OK) return st;
        L->cur = 1 - L->cur;
        L->step += 1;
    }
    return BTRT_OK;
}

btrt_status btrt_step_residual(btrt_lattice L, int64_t nsteps, double *residual) {
    NvtxRange range("btrt_step_residual");
    if (!L || !residual) return fail(BTRT_EINVAL, "null argument");
    if (!L->ready) return fail(BTRT_ESTATE, "lattice not initialised");
    if (nsteps < 1) return fail(BTRT_EINVAL, "btrt_step_residual needs at least one step");
    btrt_status st = btrt_step(L, nsteps - 1);
    if (st != BTRT_OK) return st;
    st = launch(L, L->step + 1, false, true);
    if (st != BTRT_OK) return st;
    L->cur = 1 - L->cur;
    L->step += 1;
    // fixed-order FP64 reduction of the per-block partials, then sqrt on the host
    const long long nb = L->lay.resid_blocks;
    CUDA_TRY(enqueue_rows_sum<double>(L->resid_partials(), (int)std::min<long long>(nb, 1 << 30), 1, nb,
                                      L->partials(), L->red_out(), L->stream));
    double s2 = 0.0;
    CUDA_TRY(cudaMemcpyAsync(&s2, L->red_out(), sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CUDA_TRY(cudaStreamSynchronize(L->stream));
    *residual = std::sqrt(s2);
    return BTRT_OK;
}

btrt_status btrt_read_phi(btrt_lattice L, void *dst, int32_t dtype, int32_t on_device) {
    if (!L || !dst) return fail(BTRT_EINVAL, "null argument");
    if (!L->ready) return fail(BTRT_ESTATE, "lattice not initialised");
    if (dtype != BTRT_F64 && dtype != BTRT_F32) return fail(BTRT_EINVAL, "dtype must be F64 or F32");
    return L->g.compute == BTRT_F64    ? copy_phi_out<double>(L, dst, dtype, on_device)
           : L->g.compute == BTRT_DF64 ? copy_phi_out<dw>(L, dst, dtype, on_device)
                                       : copy_phi_out<float>(L, dst, dtype, on_device);
}

btrt_status btrt_read_f(btrt_lattice L, double *dst, int32_t x0, int32_t y0, int32_t w, int32_t h) {
    if (!L || !dst) return fail(BTRT_EINVAL, "null argument");
    if (!L->ready) return fail(BTRT_ESTATE, "lattice not initialised");
    const btrt_grid_desc &g = L->g;
    if (w <= 0 || h <= 0 || x0 < 0 || y0 < 0 || x0 + w > g.nx || y0 + h > g.ny)
        return fail(BTRT_EINVAL, "window outside the grid");
    const size_t sf = elem_size(g.storage);
    std::vector<unsigned char> raw((size_t)w * h * sf);
    const double wts[9] = {4.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 9, 1.0 / 36, 1.0 / 36, 1.0 / 36, 1.0 / 36};
    // FP16 deviations of the stochastically rounded forms are stored scaled by 2^12
    const bool sr_f16 = stochastic_store(g) && g.storage == BTRT_F16;
    // the local forms: stored relative to the node's phi (both words of a double-word phi)
    const int sh0 = shift_of(g);
    const int sh = (sh0 == kShiftLocalSR || sh0 == kShiftMomentSR) ? kShiftLocal
                   : (sh0 == kShiftLocalDWSR ? kShiftLocalDW : sh0);
    std::vector<float> phiw, phiw_lo;   // the nodes' phi, for the local shifts (FP32 compute)
    std::vector<double> jxw, jyw;       // the nodes' stored first moments (BTRT_SHIFT_MOMENT_SR)
    if (has_j(g)) {
        std::vector<unsigned char> jr((size_t)w * h * sf);
        for (int c = 0; c < 2; ++c) {
            const unsigned char *src = static_cast<unsigned char *>(L->jplanes(L->cur)) +
                                       ((size_t)c * L->lay.plane + (size_t)y0 * L->lay.pitch + x0) * sf;
            CUDA_TRY(cudaMemcpy2DAsync(jr.data(), w * sf, src, L->lay.pitch * sf, w * sf, h, cudaMemcpyDeviceToHost,
                                       L->stream));
            CUDA_TRY(cudaStreamSynchronize(L->stream));
            std::vector<double> &dj = c == 0 ? jxw : jyw;
            dj.resize((size_t)w * h);
            for (size_t k = 0; k < dj.size(); ++k)
                dj[k] = half_bits_to_double(g.storage, &jr[k * 2]) * (sr_f16 ? 1.0 / 4096.0 : 1.0);
        }
    }
    if (sh == kShiftLocal || sh == kShiftLocalDW) {
        phiw.resize((size_t)w * h);
        CUDA_TRY(cudaMemcpy2DAsync(phiw.data(), w * sizeof(float), L->phi<float>() + (size_t)y0 * L->lay.pitch + x0,
                                   L->lay.pitch * sizeof(float), w * sizeof(float), h, cudaMemcpyDeviceToHost,
                                   L->stream));
        if (sh == kShiftLocalDW) {
            phiw_lo.resize((size_t)w * h);
            CUDA_TRY(cudaMemcpy2DAsync(phiw_lo.data(), w * sizeof(float),
                                       L->phi_lo(L->cur) + (size_t)y0 * L->lay.pitch + x0,
                                       L->lay.pitch * sizeof(float), w * sizeof(float), h, cudaMemcpyDeviceToHost,
                                       L->stream));
        }
        CUDA_TRY(cudaStreamSynchronize(L->stream));
    }
    for (int i = 0; i < 9; ++i) {
        const unsigned char *src = static_cast<unsigned char *>(L->fbuf(L->cur)) +
                                   ((size_t)i * L->lay.plane + (size_t)y0 * L->lay.pitch + x0) * sf;
        CUDA_TRY(cudaMemcpy2DAsync(raw.data(), w * sf, src, L->lay.pitch * sf, w * sf, h,
                                   cudaMemcpyDeviceToHost, L->stream));
        CUDA_TRY(cudaStreamSynchronize(L->stream));
        // the stored values are rounded from f - w_i phi_ref (reference shift, FP32 compute
        // shifts by (float)(w_i phi_ref)) or from f^+ - w_i phi(x) (local shift); FP64 and
        // double-word storage are never shifted
        const double shift = sh == kShiftRef ? (double)(float)(wts[i] * g.phi_ref) : 0.0;
        for (size_t k = 0; k < (size_t)w * h; ++k) {
            double v;
            if (g.storage == BTRT_F64) std::memcpy(&v, &raw[k * 8], 8);
            else if (g.storage == BTRT_DF64) {
                float hl[2];
                std::memcpy(hl, &raw[k * 8], 8);
                v = (double)hl[0] + (double)hl[1];
            }
            else if (g.storage == BTRT_F32) { float fv; std::memcpy(&fv, &raw[k * 4], 4); v = fv; }
            else v = half_bits_to_double(g.storage, &raw[k * 2]) * (sr_f16 ? 1.0 / 4096.0 : 1.0);
            double loc = sh == kShiftLocal     ? wts[i] * (double)phiw[k]
                         : sh == kShiftLocalDW ? wts[i] * ((double)phiw[k] + (double)phiw_lo[k])
                                               : 0.0;
            if (has_j(g)) loc += 3.0 * wts[i] * (ex_of(i) * jxw[k] + ey_of(i) * jyw[k]);
            dst[(size_t)i * w * h + k] = v + shift + loc;
        }
    }
    return BTRT_OK;
}

btrt_status btrt_mass(btrt_lattice L, double *out) {
    if (!L || !out) return fail(BTRT_EINVAL, "null argument");
    if (!L->ready) return fail(BTRT_ESTATE, "lattice not initialised");
    return L->g.compute == BTRT_F64    ? reduce_phi<double>(L, out)
           : L->g.compute == BTRT_DF64 ? reduce_phi<dw>(L, out)
                                       : reduce_phi<float>(L, out);
}

btrt_status btrt_check(btrt_lattice L, int32_t *flags) {
    if (!L || !flags) return fail(BTRT_EINVAL, "null argument");
    CUDA_TRY(cudaMemcpyAsync(flags, L->flags(), sizeof(int32_t), cudaMemcpyDeviceToHost, L->stream));
    CUDA_TRY(cudaStreamSynchronize(L->stream));
    if (*flags & 8) return fail(BTRT_ECUDA, "an index check of the debug build failed (flag bit 3)");
    if (*flags & 4) return fail(BTRT_ETIMEOUT, "a bounded wait for a tile copy gave up");
    if (*flags & 1) return fail(BTRT_EUNSTABLE, "non-finite phi detected (unstable parameters?)");
    return BTRT_OK;
}

btrt_status btrt_set_sweep_variant(btrt_lattice L, int32_t variant) {
    if (!L) return fail(BTRT_EINVAL, "null lattice");
    if (variant != BTRT_SWEEP_AUTO && variant != BTRT_SWEEP_PLAIN && variant != BTRT_SWEEP_TMA &&
        variant != BTRT_SWEEP_TB2 && variant != BTRT_SWEEP_VEC && variant != BTRT_SWEEP_TB2V)
        return fail(BTRT_EINVAL, "unknown sweep variant %d", variant);
    if ((variant == BTRT_SWEEP_TB2 || variant == BTRT_SWEEP_TB2V) && L->g.compute != BTRT_F32)
        return fail(BTRT_EINVAL, "the two-step sweeps serve FP32-compute lattices");
    if (variant == BTRT_SWEEP_VEC && L->g.compute != BTRT_F32)
        return fail(BTRT_EINVAL, "the vector-access sweep serves FP32-compute lattices");
    if (has_phi_lo(L->g) && variant != BTRT_SWEEP_AUTO && variant != BTRT_SWEEP_PLAIN)
        return fail(BTRT_EINVAL, "lattices with double-word phi planes (BTRT_SHIFT_LOCAL_DW, _DW_SR) take the plain form");
    if (stochastic_store(L->g) && variant != BTRT_SWEEP_AUTO && variant != BTRT_SWEEP_PLAIN &&
        variant != BTRT_SWEEP_VEC)
        return fail(BTRT_EINVAL, "stochastically rounded storage (BTRT_SHIFT_LOCAL_SR, _MOMENT_SR) takes the plain or "
                    "vector form");
    if (variant == BTRT_SWEEP_TMA && !L->have_tma)
        return fail(BTRT_EINVAL, "the TMA sweep serves FP32-compute lattices whose tensor maps could be encoded");
    L->sweep_variant = variant;
    return BTRT_OK;
}

btrt_status btrt_get_time(btrt_lattice L, int64_t *step, double *t) {
    if (!L) return fail(BTRT_EINVAL, "null lattice");
    if (step) *step = L->step;
    if (t) *t = L->t0 + (double)L->step * L->g.dt;
    return BTRT_OK;
}

// Bytes of one phi buffer (both words of a double-word phi; the first-moment planes).
static size_t phi_state_bytes(btrt_lattice L) {
    return (has_phi_lo(L->g) ? 2 : 1) * (size_t)L->lay.plane * elem_size(L->g.compute) +
           (has_j(L->g) ? 2 * (size_t)L->lay.plane * elem_size(L->g.storage) : 0);
}

size_t btrt_state_bytes(btrt_lattice L) {
    if (!L) return 0;
    return sizeof(StateHeader) + L->lay.fbuf_bytes + phi_state_bytes(L);
}

btrt_status btrt_save(btrt_lattice L, void *host_buf, size_t n) {
    if (!L || !host_buf) return fail(BTRT_EINVAL, "null argument");
    if (!L->ready) return fail(BTRT_ESTATE, "lattice not initialised");
    if (n < btrt_state_bytes(L)) return fail(BTRT_ENOMEM, "buffer of %zu bytes too small", n);
    StateHeader h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "BTRTST2", 8);
    h.shift = L->g.shift;
    h.nx = L->g.nx;
    h.ny = L->g.ny;
    h.compute = L->g.compute;
    h.storage = L->g.storage;
    h.step = L->step;
    h.t0 = L->t0;
    std::memcpy(host_buf, &h, sizeof h);
    unsigned char *p = static_cast<unsigned char *>(host_buf) + sizeof h;
    CUDA_TRY(cudaMemcpyAsync(p, L->fbuf(L->cur), L->lay.fbuf_bytes, cudaMemcpyDeviceToHost, L->stream));
    CUDA_TRY(cudaMemcpyAsync(p + L->lay.fbuf_bytes, L->ws + L->lay.off_phi[L->cur], phi_state_bytes(L),
                             cudaMemcpyDeviceToHost, L->stream));
    CUDA_TRY(cudaStreamSynchronize(L->stream));
    return BTRT_OK;
}

btrt_status btrt_load(btrt_lattice L, const void *host_buf, size_t n) {
    if (!L || !host_buf) return fail(BTRT_EINVAL, "null argument");
    if (!L->have_coeffs) return fail(BTRT_ESTATE, "btrt_set_coeffs must come before btrt_load");
    if (n < btrt_state_bytes(L)) return fail(BTRT_ENOMEM, "buffer of %zu bytes too small", n);
    StateHeader h;
    std::memcpy(&h, host_buf, sizeof h);
    if (std::memcmp(h.magic, "BTRTST2", 8) != 0 || h.nx != L->g.nx || h.ny != L->g.ny ||
        h.compute != L->g.compute || h.storage != L->g.storage || h.shift != L->g.shift)
        return fail(BTRT_EINVAL, "state does not match this lattice");
    const unsigned char *p = static_cast<const unsigned char *>(host_buf) + sizeof h;
    L->cur = 0;
    CUDA_TRY(cudaMemcpyAsync(L->fbuf(0), p, L->lay.fbuf_bytes, cudaMemcpyHostToDevice, L->stream));
    CUDA_TRY(cudaMemcpyAsync(L->ws + L->lay.off_phi[0], p + L->lay.fbuf_bytes, phi_state_bytes(L),
                             cudaMemcpyHostToDevice, L->stream));
    CUDA_TRY(cudaMemsetAsync(L->flags(), 0, 16, L->stream));
    CUDA_TRY(cudaStreamSynchronize(L->stream));
    L->step = h.step;
    L->t0 = h.t0;
    L->ready = true;
    return BTRT_OK;
}

btrt_status btrt_destroy(btrt_lattice L) {
    if (L && L->batch_refs > 0) return fail(BTRT_ESTATE, "lattice is still a member of %d batch(es)", L->batch_refs);
    delete L;
    return BTRT_OK;
}

const char *btrt_last_error(void) { return g_err.c_str(); }

const char *btrt_version(void) { return "btrt 0.1 (D2Q9 B-TriRT, sm_103a)"; }

}  // extern "C"
