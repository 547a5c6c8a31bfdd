// btrt3_api.cu -- host side of the D3Q19 C ABI (include/btrt3.h): workspace
// layout, parameter preparation, staging of phi0, reads and reductions.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstring>
#include <new>
#include <vector>

#include "../../include/btrt3.h"
#include "btrt_internal.h"
#include "btrt_launch3.cuh"

using namespace btrt;

namespace {

constexpr size_t kAlign3 = 256;

size_t up(size_t v, size_t a) { return (v + a - 1) / a * a; }

btrt_status fail3(btrt_status code, const char *msg) {
    set_last_error("%s", msg);
    return code;
}

#define CUDA3_TRY(expr)                                                                        \
    do {                                                                                       \
        cudaError_t e_ = (expr);                                                               \
        if (e_ != cudaSuccess) {                                                               \
            set_last_error("%s: %s (%s:%d)", #expr, cudaGetErrorString(e_), __FILE__, __LINE__); \
            return BTRT_ECUDA;                                                                 \
        }                                                                                      \
    } while (0)

struct Layout3 {
    long long pitch = 0, slab = 0, plane = 0;
    size_t fbuf_bytes = 0;
    size_t off_f[2] = {0, 0}, off_phi[2] = {0, 0}, off_red = 0, off_srcf = 0, total = 0;
};

btrt_status check3(const btrt3_grid_desc *g) {
    if (!g) return fail3(BTRT_EINVAL, "null grid description");
    if (g->nx < 3 || g->ny < 3 || g->nz < 3 || g->nz > 65535)
        return fail3(BTRT_EINVAL, "each of nx, ny, nz must be >= 3 (nz <= 65535)");
    for (int k = 0; k < 6; ++k)
        if (g->bc[k] != BTRT_BC_PERIODIC && g->bc[k] != BTRT_BC_HBB)
            return fail3(BTRT_EINVAL, "unknown boundary kind");
    if (g->bc[0] != g->bc[1] || g->bc[2] != g->bc[3] || g->bc[4] != g->bc[5])
        return fail3(BTRT_EINVAL, "opposite faces must share the boundary kind");
    if (g->compute == BTRT_F64) {
        if (g->storage != BTRT_F64) return fail3(BTRT_EINVAL, "FP64 compute requires FP64 storage");
    } else if (g->compute == BTRT_F32) {
        if (g->storage != BTRT_F32 && g->storage != BTRT_F16 && g->storage != BTRT_BF16)
            return fail3(BTRT_EINVAL, "FP32 compute takes F32, F16 or BF16 storage");
    } else {
        return fail3(BTRT_EINVAL, "the D3Q19 sweep computes in BTRT_F64 or BTRT_F32");
    }
    if (g->shift != BTRT_SHIFT_REF && g->shift != BTRT_SHIFT_LOCAL) return fail3(BTRT_EINVAL, "unknown storage shift");
    if (g->fields & ~BTRT_FIELD_SOURCE) return fail3(BTRT_EINVAL, "the D3Q19 lattice has only the source field");
    if (!(g->dx > 0.0) || !(g->dt > 0.0) || !std::isfinite(g->dx) || !std::isfinite(g->dt))
        return fail3(BTRT_EINVAL, "dx and dt must be positive and finite");
    if (!std::isfinite(g->phi_ref) || !std::isfinite(g->x0) || !std::isfinite(g->y0) || !std::isfinite(g->z0))
        return fail3(BTRT_EINVAL, "phi_ref, x0, y0, z0 must be finite");
    const long long pitch = (long long)((g->nx + 63) / 64) * 64;
    if (19LL * pitch * g->ny * g->nz >= (1LL << 31))
        return fail3(BTRT_EINVAL, "grid too large: 19 padded population planes must hold fewer than 2^31 values");
    return BTRT_OK;
}

Layout3 layout3(const btrt3_grid_desc *g) {
    Layout3 L;
    const size_t sf = elem_size(g->storage), sr = elem_size(g->compute);
    L.pitch = (long long)up((size_t)g->nx, 64);
    L.slab = L.pitch * g->ny;
    L.plane = L.slab * g->nz;
    L.fbuf_bytes = up(19 * (size_t)L.plane * sf, kAlign3);
    size_t off = 0;
    for (int k = 0; k < 2; ++k) {
        L.off_f[k] = off;
        off += L.fbuf_bytes;
    }
    for (int k = 0; k < 2; ++k) {
        L.off_phi[k] = off;
        off += up((size_t)L.plane * sr, kAlign3);
    }
    L.off_red = off;
    off += up((kRedBlocks + 2) * sizeof(double) + 16, kAlign3);
    if (g->fields & BTRT_FIELD_SOURCE) {
        L.off_srcf = off;
        off += up((size_t)L.plane * sr, kAlign3);
    }
    L.total = off;
    return L;
}

// rows = ny * nz rows of nx values, pitched
template <typename Real, typename In>
__global__ void dense_to_planes3(const In *__restrict__ src, Real *__restrict__ dst, int nx, long long rows,
                                 long long pitch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    for (long long r = blockIdx.y; r < rows; r += gridDim.y)
        if (x < nx) dst[r * pitch + x] = Real((double)src[r * nx + x]);
}

template <typename Real, typename Out>
__global__ void planes_to_dense3(const Real *__restrict__ src, Out *__restrict__ dst, int nx, long long rows,
                                 long long pitch) {
    const int x = blockIdx.x * blockDim.x + threadIdx.x;
    for (long long r = blockIdx.y; r < rows; r += gridDim.y)
        if (x < nx) dst[r * nx + x] = (Out)(double)src[r * pitch + x];
}

}  // namespace

struct btrt3_lattice_s {
    btrt3_grid_desc g;
    btrt3_coeffs c;
    Layout3 lay;
    unsigned char *ws = nullptr;
    cudaStream_t stream = nullptr;
    int cur = 0;
    int64_t step = 0;
    double t0 = 0.0;
    bool have_coeffs = false, ready = false, have_srcf = false;
    // lattice-unit constants
    double u[3] = {0, 0, 0}, bg[3] = {0, 0, 0}, bq = 2, A0[6] = {0, 0, 0, 0, 0, 0}, K1[6] = {0, 0, 0, 0, 0, 0},
           k2 = 1;
    bool nonlin = false;

    void *fbuf(int k) { return ws + lay.off_f[k]; }
    template <typename Real> Real *phi(int k) { return reinterpret_cast<Real *>(ws + lay.off_phi[k]); }
    double *partials() { return reinterpret_cast<double *>(ws + lay.off_red); }
    double *red_out() { return partials() + kRedBlocks; }
    int *flags() { return reinterpret_cast<int *>(partials() + kRedBlocks + 2); }
    template <typename Real> Real *srcf() {
        return lay.off_srcf ? reinterpret_cast<Real *>(ws + lay.off_srcf) : nullptr;
    }
    long long rows() const { return (long long)g.ny * g.nz; }
};

namespace {

void step_scalars3(btrt3_lattice L, int64_t n, bool first, double *src_val, double *wall_fac) {
    const double tn = L->t0 + (double)n * L->g.dt;
    *wall_fac = L->c.wall_lam == 0.0 ? 1.0 : std::exp(L->c.wall_lam * tn);
    switch (L->c.src_kind) {
    case BTRT_SRC_CONST: *src_val = L->c.src_const * L->g.dt; break;
    case BTRT_SRC_REACTION: *src_val = L->g.dt; break;
    case BTRT_SRC_FIELD: {
        const double Tn = std::exp(L->c.src_lam * tn);
        const double Tp = first ? Tn : std::exp(L->c.src_lam * (tn - L->g.dt));
        *src_val = L->g.dt * 0.5 * (3.0 * Tn - Tp);
        break;
    }
    default: *src_val = 0.0;
    }
}

int mode3(btrt3_lattice L) {
    const btrt3_coeffs &c = L->c;
    if (c.b2 != 0.0 || c.c3 != 0.0 || c.a2 != 0.0) return kGeneral;
    return c.k0 == 1.0 ? kLinearK0One : kLinear;
}

template <typename Real>
void fill3(btrt3_lattice L, Sweep3Params<Real> &p, int64_t n, bool first) {
    const btrt3_grid_desc &g = L->g;
    const btrt3_coeffs &c = L->c;
    std::memset(&p, 0, sizeof p);
    p.fin = L->fbuf(L->cur);
    p.fout = L->fbuf(first ? L->cur : 1 - L->cur);
    p.phi_in = L->phi<Real>(L->cur);
    p.phi_out = L->phi<Real>(first ? L->cur : 1 - L->cur);
    p.nx = g.nx;
    p.ny = g.ny;
    p.nz = g.nz;
    p.pitch = (int)L->lay.pitch;
    p.slab = (int)L->lay.slab;
    p.plane = (int)L->lay.plane;
    p.hbb_x = g.bc[0] == BTRT_BC_HBB;
    p.hbb_y = g.bc[2] == BTRT_BC_HBB;
    p.hbb_z = g.bc[4] == BTRT_BC_HBB;
    double sv = 0.0, wf = 1.0;
    step_scalars3(L, n, first, &sv, &wf);
    for (int k = 0; k < 6; ++k) p.wall[k] = (Real)c.wall[k];
    p.wall_fac = (Real)wf;
    const bool ref = g.storage != BTRT_F64 && g.shift == BTRT_SHIFT_REF;
    const double w3[3] = {1.0 / 3.0, 1.0 / 18.0, 1.0 / 36.0};
    for (int k = 0; k < 3; ++k) p.wref[k] = ref ? (Real)(w3[k] * g.phi_ref) : (Real)0.0;
    p.phi_ref = ref ? (Real)g.phi_ref : (Real)0.0;
    p.ux = (Real)L->u[0];
    p.uy = (Real)L->u[1];
    p.uz = (Real)L->u[2];
    p.bgx = (Real)L->bg[0];
    p.bgy = (Real)L->bg[1];
    p.bgz = (Real)L->bg[2];
    p.bq = (Real)L->bq;
    p.bq2 = L->bq == 2.0 ? 1 : 0;
    p.c3 = (Real)c.c3;
    for (int k = 0; k < 6; ++k) {
        p.A0[k] = (Real)L->A0[k];
        p.K1[k] = (Real)L->K1[k];
    }
    {
        // constant-coefficient fold: K1 u and (I - K1/2) u
        const double *K = L->K1, *u = L->u;
        const double Ku[3] = {K[0] * u[0] + K[1] * u[1] + K[2] * u[2], K[1] * u[0] + K[3] * u[1] + K[4] * u[2],
                              K[2] * u[0] + K[4] * u[1] + K[5] * u[2]};
        for (int k = 0; k < 3; ++k) {
            p.Ku[k] = (Real)Ku[k];
            p.gu[k] = (Real)(u[k] - 0.5 * Ku[k]);
        }
    }
    p.a2 = (Real)c.a2;
    p.k0 = (Real)c.k0;
    p.om = (Real)(1.0 - c.k0);
    p.nonlin = L->nonlin ? 1 : 0;
    p.k2_hbb = c.k2_mode == BTRT_K2_HBB;
    p.k2c = (Real)c.k2;
    p.k2 = (Real)L->k2;
    {
        const double k0 = c.k0, dk = L->k2 - k0;
        p.Q[0] = (Real)(L->K1[0] - k0);
        p.Q[1] = (Real)(L->K1[3] - k0);
        p.Q[2] = (Real)(L->K1[5] - k0);
        p.ka[0] = (Real)(1.5 * dk);
        p.ka[1] = (Real)(0.25 * dk);
        p.ka[2] = (Real)(0.125 * dk);
        p.kak[0] = (Real)(-1.5 * k0);
        p.kak[1] = (Real)(-0.25 * k0);
        p.kak[2] = (Real)(-0.125 * k0);
        p.a2x3 = (Real)(3.0 * c.a2);
        p.k0x15 = (Real)(1.5 * k0);
        p.k0_one = k0 == 1.0 ? 1 : 0;
    }
    p.cond_limit = (Real)1.0e6;
    for (int k = 0; k < 6; ++k) p.A0d[k] = L->A0[k];
    p.a2d = c.a2;
    p.src_kind = c.src_kind;
    p.src_val = (Real)sv;
    p.srcF = L->srcf<Real>();
    p.react_rate = (Real)c.react_rate;
    p.react_exp = (Real)c.react_exp;
    p.react2 = c.react_exp == 2.0 ? 1 : 0;
    half_split(L->bq, &p.bq_n, &p.bq_h);
    half_split(c.react_exp, &p.re_n, &p.re_h);
    p.first = first ? 1 : 0;
    p.flags = L->flags();
}

btrt_status launch3(btrt3_lattice L, int64_t n, bool first) {
    if (L->g.compute == BTRT_F64) {
        Sweep3Params<double> p;
        fill3(L, p, n, first);
        CUDA3_TRY(launch_sweep3_f64(p, mode3(L), L->stream));
    } else {
        Sweep3Params<float> p;
        fill3(L, p, n, first);
        const int sh = L->g.shift == BTRT_SHIFT_LOCAL ? kShiftLocal : kShiftRef;
        CUDA3_TRY(launch_sweep3_f32(p, L->g.storage, sh, mode3(L), L->stream));
    }
    return BTRT_OK;
}

template <typename Real>
btrt_status stage3(btrt3_lattice L, const void *phi0, int dtype, int on_device) {
    const size_t n = (size_t)L->g.nx * L->g.ny * L->g.nz;
    const size_t bytes = n * elem_size(dtype);
    const void *src = phi0;
    if (!on_device) {
        if (bytes > L->lay.fbuf_bytes) return fail3(BTRT_ENOMEM, "staging area too small");
        CUDA3_TRY(cudaMemcpyAsync(L->fbuf(1), phi0, bytes, cudaMemcpyHostToDevice, L->stream));
        src = L->fbuf(1);
    }
    const dim3 blk(256), grd((unsigned)((L->g.nx + 255) / 256), (unsigned)std::min<long long>(L->rows(), 65535));
    if (dtype == BTRT_F64)
        dense_to_planes3<Real, double><<<grd, blk, 0, L->stream>>>((const double *)src, L->phi<Real>(0), L->g.nx,
                                                                    L->rows(), L->lay.pitch);
    else
        dense_to_planes3<Real, float><<<grd, blk, 0, L->stream>>>((const float *)src, L->phi<Real>(0), L->g.nx,
                                                                   L->rows(), L->lay.pitch);
    CUDA3_TRY(cudaGetLastError());
    if (!on_device) CUDA3_TRY(cudaStreamSynchronize(L->stream));
    return BTRT_OK;
}

template <typename Real>
btrt_status read3(btrt3_lattice L, void *dst, int dtype, int on_device) {
    const size_t n = (size_t)L->g.nx * L->g.ny * L->g.nz;
    const dim3 blk(256), grd((unsigned)((L->g.nx + 255) / 256), (unsigned)std::min<long long>(L->rows(), 65535));
    if (on_device) {
        if (dtype == BTRT_F64)
            planes_to_dense3<Real, double><<<grd, blk, 0, L->stream>>>(L->phi<Real>(L->cur), (double *)dst, L->g.nx,
                                                                        L->rows(), L->lay.pitch);
        else
            planes_to_dense3<Real, float><<<grd, blk, 0, L->stream>>>(L->phi<Real>(L->cur), (float *)dst, L->g.nx,
                                                                       L->rows(), L->lay.pitch);
        CUDA3_TRY(cudaGetLastError());
        return BTRT_OK;
    }
    std::vector<Real> h(n);
    CUDA3_TRY(cudaMemcpy2DAsync(h.data(), L->g.nx * sizeof(Real), L->phi<Real>(L->cur), L->lay.pitch * sizeof(Real),
                                L->g.nx * sizeof(Real), (size_t)L->rows(), cudaMemcpyDeviceToHost, L->stream));
    CUDA3_TRY(cudaStreamSynchronize(L->stream));
    if (dtype == BTRT_F64)
        for (size_t k = 0; k < n; ++k) ((double *)dst)[k] = (double)h[k];
    else
        for (size_t k = 0; k < n; ++k) ((float *)dst)[k] = (float)h[k];
    return BTRT_OK;
}

template <typename Real>
btrt_status mass3(btrt3_lattice L, double *out) {
    CUDA3_TRY(enqueue_rows_sum<Real>(L->phi<Real>(L->cur), L->g.nx, L->rows(), L->lay.pitch, L->partials(),
                                     L->red_out(), L->stream));
    CUDA3_TRY(cudaMemcpyAsync(out, L->red_out(), sizeof(double), cudaMemcpyDeviceToHost, L->stream));
    CUDA3_TRY(cudaStreamSynchronize(L->stream));
    return BTRT_OK;
}


}  // namespace

extern "C" {

size_t btrt3_workspace_bytes(const btrt3_grid_desc *g) {
    if (check3(g) != BTRT_OK) return 0;
    return layout3(g).total;
}

btrt_status btrt3_create(const btrt3_grid_desc *g, void *dev_workspace, size_t workspace_bytes, void *cuda_stream,
                         btrt3_lattice *out) {
    if (!out) return fail3(BTRT_EINVAL, "null output handle");
    *out = nullptr;
    btrt_status st = check3(g);
    if (st != BTRT_OK) return st;
    if (!dev_workspace) return fail3(BTRT_EINVAL, "null workspace");
    if ((uintptr_t)dev_workspace % kAlign3) return fail3(BTRT_EINVAL, "workspace not 256-byte aligned");
    const Layout3 lay = layout3(g);
    if (workspace_bytes < lay.total) return fail3(BTRT_ENOMEM, "workspace too small");
    cudaPointerAttributes attr;
    if (cudaPointerGetAttributes(&attr, dev_workspace) != cudaSuccess || attr.type != cudaMemoryTypeDevice) {
        cudaGetLastError();
        return fail3(BTRT_EINVAL, "workspace is not device memory");
    }
    btrt3_lattice L = new (std::nothrow) btrt3_lattice_s();
    if (!L) return fail3(BTRT_ENOMEM, "host allocation failed");
    L->g = *g;
    L->lay = lay;
    L->ws = static_cast<unsigned char *>(dev_workspace);
    L->stream = static_cast<cudaStream_t>(cuda_stream);
    std::memset(&L->c, 0, sizeof L->c);
    L->c.k0 = 1.0;
    if (cudaMemsetAsync(L->flags(), 0, 16, L->stream) != cudaSuccess) {
        delete L;
        return fail3(BTRT_ECUDA, "cudaMemsetAsync failed");
    }
    *out = L;
    return BTRT_OK;
}

btrt_status btrt3_set_coeffs(btrt3_lattice L, const btrt3_coeffs *c) {
    if (!L || !c) return fail3(BTRT_EINVAL, "null argument");
    const double *a = c->A0;
    // SPD by leading principal minors
    const double m1 = a[0], m2 = a[0] * a[3] - a[1] * a[1];
    const double m3 = a[0] * (a[3] * a[5] - a[4] * a[4]) - a[1] * (a[1] * a[5] - a[4] * a[2]) +
                      a[2] * (a[1] * a[4] - a[3] * a[2]);
    if (!(m1 > 0.0 && m2 > 0.0 && m3 > 0.0)) return fail3(BTRT_EINVAL, "A0 must be symmetric positive definite");
    if (!(c->k0 > 0.0 && c->k0 < 2.0)) return fail3(BTRT_EINVAL, "k0 outside (0, 2)");
    if (c->k2_mode != BTRT_K2_HBB && c->k2_mode != BTRT_K2_CONST) return fail3(BTRT_EINVAL, "unknown k2 mode");
    if (c->k2_mode == BTRT_K2_CONST && !(c->k2 > 0.0 && c->k2 < 2.0)) return fail3(BTRT_EINVAL, "k2 outside (0, 2)");
    if (c->src_kind != BTRT_SRC_NONE && c->src_kind != BTRT_SRC_CONST && c->src_kind != BTRT_SRC_FIELD &&
        c->src_kind != BTRT_SRC_REACTION)
        return fail3(BTRT_EINVAL, "the D3Q19 lattice takes source kinds NONE, CONST, FIELD, REACTION");
    if (c->src_kind == BTRT_SRC_FIELD && !(L->g.fields & BTRT_FIELD_SOURCE))
        return fail3(BTRT_EINVAL, "BTRT_SRC_FIELD needs BTRT_FIELD_SOURCE in the grid description");
    if (c->src_kind == BTRT_SRC_REACTION && (!std::isfinite(c->react_rate) || !(c->react_exp > 0.0)))
        return fail3(BTRT_EINVAL, "reaction source needs a finite rate and an exponent > 0");
    if (!(c->b_q == 0.0 || (c->b_q >= 1.0 && std::isfinite(c->b_q))))
        return fail3(BTRT_EINVAL, "flux exponent must be 0 (default 2) or >= 1");
    if (!std::isfinite(c->a2) || c->a2 < 0.0) return fail3(BTRT_EINVAL, "a2 must be >= 0");
    for (int k = 0; k < 6; ++k)
        if (!std::isfinite(c->wall[k])) return fail3(BTRT_EINVAL, "non-finite wall value");
    L->c = *c;
    const double cl = L->g.dx / L->g.dt, sA = L->g.dt / (L->g.dx * L->g.dx);
    const bool dflt = c->b_dir[0] == 0.0 && c->b_dir[1] == 0.0 && c->b_dir[2] == 0.0;
    const double q = c->b_q == 0.0 ? 2.0 : c->b_q;
    L->bq = q;
    for (int k = 0; k < 3; ++k) {
        L->u[k] = c->u[k] / cl;
        L->bg[k] = (c->b2 / cl) * (dflt ? 1.0 : c->b_dir[k]) / q;
    }
    for (int k = 0; k < 6; ++k) L->A0[k] = a[k] * sA;
    // K1 = (3 A^ + I/2)^{-1} at A0 (Eq. 30), symmetric, by cofactors; k2 from Eq. 62 at k1_eff = 3 / tr
    const double *A = L->A0;
    const double mxx = 3 * A[0] + 0.5, mxy = 3 * A[1], mxz = 3 * A[2], myy = 3 * A[3] + 0.5, myz = 3 * A[4],
                 mzz = 3 * A[5] + 0.5;
    const double cxx = myy * mzz - myz * myz, cxy = mxz * myz - mxy * mzz, cxz = mxy * myz - mxz * myy;
    const double cyy = mxx * mzz - mxz * mxz, cyz = mxy * mxz - mxx * myz, czz = mxx * myy - mxy * mxy;
    const double det = mxx * cxx + mxy * cxy + mxz * cxz;
    L->K1[0] = cxx / det;
    L->K1[1] = cxy / det;
    L->K1[2] = cxz / det;
    L->K1[3] = cyy / det;
    L->K1[4] = cyz / det;
    L->K1[5] = czz / det;
    const double k1eff = 3.0 / (mxx + myy + mzz);
    L->k2 = c->k2_mode == BTRT_K2_HBB ? 8.0 * (k1eff - 2.0) / (3.0 * (k1eff - 4.0)) : c->k2;
    L->nonlin = c->a2 != 0.0;
    L->have_coeffs = true;
    return BTRT_OK;
}

btrt_status btrt3_set_source_field(btrt3_lattice L, const double *F) {
    if (!L || !F) return fail3(BTRT_EINVAL, "null argument");
    if (!(L->g.fields & BTRT_FIELD_SOURCE)) return fail3(BTRT_EINVAL, "lattice has no source-field plane");
    const size_t n = (size_t)L->g.nx * L->g.ny * L->g.nz;
    for (size_t k = 0; k < n; ++k)
        if (!std::isfinite(F[k])) return fail3(BTRT_EINVAL, "non-finite source value");
    const size_t sr = elem_size(L->g.compute);
    std::vector<unsigned char> h((size_t)L->lay.plane * sr, 0);
    for (long long r = 0; r < L->rows(); ++r)
        for (int x = 0; x < L->g.nx; ++x) {
            const double v = F[(size_t)r * L->g.nx + x];
            unsigned char *dst = h.data() + ((size_t)r * L->lay.pitch + x) * sr;
            if (sr == 8) std::memcpy(dst, &v, 8);
            else {
                const float f = (float)v;
                std::memcpy(dst, &f, 4);
            }
        }
    CUDA3_TRY(cudaMemcpyAsync(L->ws + L->lay.off_srcf, h.data(), h.size(), cudaMemcpyHostToDevice, L->stream));
    CUDA3_TRY(cudaStreamSynchronize(L->stream));
    L->have_srcf = true;
    return BTRT_OK;
}

btrt_status btrt3_init_phi(btrt3_lattice L, const void *phi0, int32_t dtype, int32_t on_device, double t0) {
    NvtxRange range("btrt3_init_phi");
    if (!L || !phi0) return fail3(BTRT_EINVAL, "null argument");
    if (!L->have_coeffs) return fail3(BTRT_ESTATE, "btrt3_set_coeffs must come before btrt3_init_phi");
    if (L->c.src_kind == BTRT_SRC_FIELD && !L->have_srcf)
        return fail3(BTRT_ESTATE, "btrt3_set_source_field must come before btrt3_init_phi");
    if (dtype != BTRT_F64 && dtype != BTRT_F32) return fail3(BTRT_EINVAL, "phi0 dtype must be F64 or F32");
    if (!std::isfinite(t0)) return fail3(BTRT_EINVAL, "t0 must be finite");
    btrt_status st = L->g.compute == BTRT_F64 ? stage3<double>(L, phi0, dtype, on_device)
                                              : stage3<float>(L, phi0, dtype, on_device);
    if (st != BTRT_OK) return st;
    L->t0 = t0;
    L->step = 0;
    L->cur = 0;
    CUDA3_TRY(cudaMemsetAsync(L->flags(), 0, 16, L->stream));
    st = launch3(L, 0, true);
    if (st != BTRT_OK) return st;
    L->ready = true;
    return BTRT_OK;
}

btrt_status btrt3_step(btrt3_lattice L, int64_t nsteps) {
    NvtxRange range("btrt3_step");
    if (!L) return fail3(BTRT_EINVAL, "null lattice");
    if (!L->ready) return fail3(BTRT_ESTATE, "lattice not initialised");
    if (nsteps < 0) return fail3(BTRT_EINVAL, "negative step count");
    for (int64_t k = 0; k < nsteps; ++k) {
        btrt_status st = launch3(L, L->step + 1, false);
        if (st != BTRT_OK) return st;
        L->cur = 1 - L->cur;
        L->step += 1;
    }
    return BTRT_OK;
}

btrt_status btrt3_read_phi(btrt3_lattice L, void *dst, int32_t dtype, int32_t on_device) {
    if (!L || !dst) return fail3(BTRT_EINVAL, "null argument");
    if (!L->ready) return fail3(BTRT_ESTATE, "lattice not initialised");
    if (dtype != BTRT_F64 && dtype != BTRT_F32) return fail3(BTRT_EINVAL, "dtype must be F64 or F32");
    return L->g.compute == BTRT_F64 ? read3<double>(L, dst, dtype, on_device) : read3<float>(L, dst, dtype, on_device);
}

btrt_status btrt3_read_f(btrt3_lattice L, double *dst, int32_t x0, int32_t y0, int32_t z0, int32_t w, int32_t h,
                         int32_t d) {
    if (!L || !dst) return fail3(BTRT_EINVAL, "null argument");
    if (!L->ready) return fail3(BTRT_ESTATE, "lattice not initialised");
    const btrt3_grid_desc &g = L->g;
    if (w <= 0 || h <= 0 || d <= 0 || x0 < 0 || y0 < 0 || z0 < 0 || x0 + w > g.nx || y0 + h > g.ny || z0 + d > g.nz)
        return fail3(BTRT_EINVAL, "box outside the grid");
    const size_t sf = elem_size(g.storage);
    const size_t cnt = (size_t)w * h * d;
    std::vector<unsigned char> raw(cnt * sf);
    std::vector<double> phiw(cnt, 0.0);
    const bool local = g.storage != BTRT_F64 && g.shift == BTRT_SHIFT_LOCAL;
    const bool ref = g.storage != BTRT_F64 && g.shift == BTRT_SHIFT_REF;
    if (local) {
        std::vector<float> pf(cnt);
        for (int z = 0; z < d; ++z)
            CUDA3_TRY(cudaMemcpy2DAsync(pf.data() + (size_t)z * w * h, w * sizeof(float),
                                        L->phi<float>(L->cur) + (size_t)(z0 + z) * L->lay.slab +
                                            (size_t)y0 * L->lay.pitch + x0,
                                        L->lay.pitch * sizeof(float), w * sizeof(float), h,
                                        cudaMemcpyDeviceToHost, L->stream));
        CUDA3_TRY(cudaStreamSynchronize(L->stream));
        for (size_t k = 0; k < cnt; ++k) phiw[k] = pf[k];
    }
    for (int i = 0; i < 19; ++i) {
        const int n2 = (cx3(i) != 0) + (cy3(i) != 0) + (cz3(i) != 0);
        const double wi = n2 == 0 ? 1.0 / 3.0 : (n2 == 1 ? 1.0 / 18.0 : 1.0 / 36.0);
        for (int z = 0; z < d; ++z) {
            const unsigned char *src = static_cast<unsigned char *>(L->fbuf(L->cur)) +
                                       ((size_t)i * L->lay.plane + (size_t)(z0 + z) * L->lay.slab +
                                        (size_t)y0 * L->lay.pitch + x0) * sf;
            CUDA3_TRY(cudaMemcpy2DAsync(raw.data() + (size_t)z * w * h * sf, w * sf, src, L->lay.pitch * sf, w * sf, h,
                                        cudaMemcpyDeviceToHost, L->stream));
        }
        CUDA3_TRY(cudaStreamSynchronize(L->stream));
        const double shift = ref ? (double)(float)(wi * g.phi_ref) : 0.0;
        for (size_t k = 0; k < cnt; ++k) {
            double v;
            if (g.storage == BTRT_F64) std::memcpy(&v, &raw[k * 8], 8);
            else if (g.storage == BTRT_F32) {
                float f;
                std::memcpy(&f, &raw[k * 4], 4);
                v = f;
            } else v = half_bits_to_double(g.storage, &raw[k * 2]);
            dst[(size_t)i * cnt + k] = v + shift + (local ? wi * phiw[k] : 0.0);
        }
    }
    return BTRT_OK;
}

btrt_status btrt3_mass(btrt3_lattice L, double *out) {
    if (!L || !out) return fail3(BTRT_EINVAL, "null argument");
    if (!L->ready) return fail3(BTRT_ESTATE, "lattice not initialised");
    return L->g.compute == BTRT_F64 ? mass3<double>(L, out) : mass3<float>(L, out);
}

btrt_status btrt3_check(btrt3_lattice L, int32_t *flags) {
    if (!L || !flags) return fail3(BTRT_EINVAL, "null argument");
    CUDA3_TRY(cudaMemcpyAsync(flags, L->flags(), sizeof(int32_t), cudaMemcpyDeviceToHost, L->stream));
    CUDA3_TRY(cudaStreamSynchronize(L->stream));
    if (*flags & 8) return fail3(BTRT_ECUDA, "an index check of the debug build failed (flag bit 3)");
    if (*flags & 1) return fail3(BTRT_EUNSTABLE, "non-finite phi detected (unstable parameters?)");
    return BTRT_OK;
}

namespace {
struct State3Header {
    char magic[8];
    int32_t nx, ny, nz, compute, storage, shift;
    int64_t step;
    double t0;
};
}  // namespace

size_t btrt3_state_bytes(btrt3_lattice L) {
    if (!L) return 0;
    return sizeof(State3Header) + L->lay.fbuf_bytes + (size_t)L->lay.plane * elem_size(L->g.compute);
}

btrt_status btrt3_save(btrt3_lattice L, void *host_buf, size_t n) {
    if (!L || !host_buf) return fail3(BTRT_EINVAL, "null argument");
    if (!L->ready) return fail3(BTRT_ESTATE, "lattice not initialised");
    if (n < btrt3_state_bytes(L)) return fail3(BTRT_ENOMEM, "buffer too small");
    State3Header h;
    std::memset(&h, 0, sizeof h);
    std::memcpy(h.magic, "BTRT3S1", 8);
    h.nx = L->g.nx;
    h.ny = L->g.ny;
    h.nz = L->g.nz;
    h.compute = L->g.compute;
    h.storage = L->g.storage;
    h.shift = L->g.shift;
    h.step = L->step;
    h.t0 = L->t0;
    std::memcpy(host_buf, &h, sizeof h);
    unsigned char *p = static_cast<unsigned char *>(host_buf) + sizeof h;
    CUDA3_TRY(cudaMemcpyAsync(p, L->fbuf(L->cur), L->lay.fbuf_bytes, cudaMemcpyDeviceToHost, L->stream));
    CUDA3_TRY(cudaMemcpyAsync(p + L->lay.fbuf_bytes, L->ws + L->lay.off_phi[L->cur],
                              (size_t)L->lay.plane * elem_size(L->g.compute), cudaMemcpyDeviceToHost, L->stream));
    CUDA3_TRY(cudaStreamSynchronize(L->stream));
    return BTRT_OK;
}

btrt_status btrt3_load(btrt3_lattice L, const void *host_buf, size_t n) {
    if (!L || !host_buf) return fail3(BTRT_EINVAL, "null argument");
    if (!L->have_coeffs) return fail3(BTRT_ESTATE, "btrt3_set_coeffs must come before btrt3_load");
    if (n < btrt3_state_bytes(L)) return fail3(BTRT_ENOMEM, "buffer too small");
    State3Header h;
    std::memcpy(&h, host_buf, sizeof h);
    if (std::memcmp(h.magic, "BTRT3S1", 8) != 0 || h.nx != L->g.nx || h.ny != L->g.ny || h.nz != L->g.nz ||
        h.compute != L->g.compute || h.storage != L->g.storage || h.shift != L->g.shift)
        return fail3(BTRT_EINVAL, "state does not match this lattice");
    const unsigned char *p = static_cast<const unsigned char *>(host_buf) + sizeof h;
    L->cur = 0;
    CUDA3_TRY(cudaMemcpyAsync(L->fbuf(0), p, L->lay.fbuf_bytes, cudaMemcpyHostToDevice, L->stream));
    CUDA3_TRY(cudaMemcpyAsync(L->ws + L->lay.off_phi[0], p + L->lay.fbuf_bytes,
                              (size_t)L->lay.plane * elem_size(L->g.compute), cudaMemcpyHostToDevice, L->stream));
    CUDA3_TRY(cudaMemsetAsync(L->flags(), 0, 16, L->stream));
    CUDA3_TRY(cudaStreamSynchronize(L->stream));
    L->step = h.step;
    L->t0 = h.t0;
    L->ready = true;
    return BTRT_OK;
}

btrt_status btrt3_get_time(btrt3_lattice L, int64_t *step, double *t) {
    if (!L) return fail3(BTRT_EINVAL, "null lattice");
    if (step) *step = L->step;
    if (t) *t = L->t0 + (double)L->step * L->g.dt;
    return BTRT_OK;
}

btrt_status btrt3_destroy(btrt3_lattice L) {
    delete L;
    return BTRT_OK;
}

}  // extern "C"
