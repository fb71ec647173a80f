// extern "C" entry points of the SIP-DG Stokes library: argument checks,
// error translation, and dispatch to the kernels.  No C++ exception leaves
// this file.
#include <cstring>

#include "sip_internal.h"

using sip::Error;

namespace {

template <typename F>
sip_status guarded(sip_ctx* ctx, F&& f) {
    try {
        f();
        if (ctx) ctx->err.clear();
        return SIP_OK;
    } catch (const Error& e) {
        if (ctx) ctx->err = e.what();
        return e.status;
    } catch (const std::bad_alloc&) {
        if (ctx) ctx->err = "host allocation failed";
        return SIP_ERR_OOM;
    } catch (const std::exception& e) {
        if (ctx) ctx->err = e.what();
        return SIP_ERR_CUDA;
    }
}

inline cudaStream_t as_stream(void* s) { return static_cast<cudaStream_t>(s); }


}  // namespace

int64_t sip_problem::device_bytes() const {
    return int64_t(eta_d.bytes + eta_f.bytes);
}

extern "C" {

void sip_problem_desc_default(sip_problem_desc* d) {
    if (!d) return;
    std::memset(d, 0, sizeof(*d));
    d->nx = d->ny = 1;
    d->lx = d->ly = 1.0;
    d->k = 2;
    for (int i = 0; i < 4; ++i) d->bc[i] = SIP_BC_NAVIER;
    d->eta_host = nullptr;
    d->penalty_scale = 1.0;
    d->n_hlevels = 0;
    d->cheb_steps_p = 2;
    d->cheb_steps_h = 3;
    d->eig_iters = 10;
    d->cheb_lo = 0.1;
    d->cheb_hi = 1.1;
    d->seed = 0;
    d->precision = SIP_PREC_FP64;
}

sip_status sip_ctx_create(int device, sip_ctx** out) {
    if (!out) return SIP_ERR_INVALID_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) {
        cudaGetLastError();
        return device < 0 ? SIP_ERR_INVALID_ARG : SIP_ERR_CUDA;
    }
    sip_ctx* c = new (std::nothrow) sip_ctx();
    if (!c) return SIP_ERR_OOM;
    c->device = device;
    if (cudaSetDevice(device) != cudaSuccess) {
        delete c;
        return SIP_ERR_CUDA;
    }
    *out = c;
    return SIP_OK;
}

void sip_ctx_destroy(sip_ctx* ctx) { delete ctx; }

const char* sip_last_error(const sip_ctx* ctx) {
    if (!ctx) return "null context";
    return ctx->err.c_str();
}

sip_status sip_problem_create(sip_ctx* ctx, const sip_problem_desc* d, sip_problem** out) {
    if (!ctx) return SIP_ERR_INVALID_ARG;
    return guarded(ctx, [&] {
        sip::require(out != nullptr && d != nullptr, "null argument");
        *out = nullptr;
        sip::require(d->nx >= 1 && d->ny >= 1, "nx and ny must be >= 1");
        sip::require(d->k >= 1 && d->k <= 6, "k must be in 1..6");
        sip::require(std::isfinite(d->lx) && std::isfinite(d->ly) && d->lx > 0 && d->ly > 0,
                     "domain lengths must be finite and positive");
        sip::require(std::isfinite(d->penalty_scale) && d->penalty_scale > 0,
                     "penalty_scale must be finite and positive");
        for (int i = 0; i < 4; ++i)
            sip::require(d->bc[i] >= SIP_BC_NAVIER && d->bc[i] <= SIP_BC_DIRICHLET,
                         "unknown boundary condition");
        sip::require(d->eta_host != nullptr, "eta_host is null");
        sip::require(d->n_hlevels >= 0, "n_hlevels must be >= 0");
        {
            int cx = d->nx, cy = d->ny;
            for (int l = 0; l < d->n_hlevels; ++l) {
                sip::require(cx % 2 == 0 && cy % 2 == 0,
                             "mesh cannot be coarsened n_hlevels times");
                cx /= 2;
                cy /= 2;
            }
        }
        const int64_t ne = int64_t(d->nx) * d->ny;
        sip::require(ne <= (int64_t(1) << 31) / 128, "mesh too large");
        std::vector<double> eta(d->eta_host, d->eta_host + ne);
        for (double v : eta)
            sip::require(std::isfinite(v) && v > 0.0, "eta must be finite and positive");
        SIP_CUDA(cudaSetDevice(ctx->device));
        auto* p = new sip_problem();
        try {
            p->ctx = ctx;
            p->desc = *d;
            p->desc.eta_host = nullptr;
            p->k = d->k;
            p->n = d->k + 1;
            p->nb = 2 * p->n * p->n;
            p->mp = d->k * d->k;
            p->ne = ne;
            p->n_u = ne * p->nb;
            p->n_p = ne * p->mp;
            p->geom = sip::make_geom(d->nx, d->ny, d->lx, d->ly, d->bc, d->k, d->penalty_scale);
            p->geom1 = p->geom;   // the Galerkin A_1 keeps the fine-k penalty
            p->eta_host = eta;
            p->eta_d.alloc(ne * sizeof(double));
            p->eta_f.alloc(ne * sizeof(float));
            std::vector<float> ef(eta.begin(), eta.end());
            SIP_CUDA(cudaMemcpy(p->eta_d.ptr, eta.data(), ne * sizeof(double),
                                cudaMemcpyHostToDevice));
            SIP_CUDA(cudaMemcpy(p->eta_f.ptr, ef.data(), ne * sizeof(float),
                                cudaMemcpyHostToDevice));
        } catch (...) {
            delete p;
            throw;
        }
        *out = p;
    });
}

void sip_problem_destroy(sip_problem* p) { delete p; }

sip_status sip_problem_sizes(const sip_problem* p, int64_t* n_u, int64_t* n_p,
                             int64_t* device_bytes) {
    if (!p) return SIP_ERR_INVALID_ARG;
    if (n_u) *n_u = p->n_u;
    if (n_p) *n_p = p->n_p;
    if (device_bytes) *device_bytes = p->device_bytes();
    return SIP_OK;
}

sip_status sip_apply_A(sip_problem* p, const double* x, double* y, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded(p->ctx, [&] {
        sip::require(x && y, "null vector");
        sip::require(x != y, "x and y must not overlap");
        sip::launch_apply_sip<double>(p->n, p->geom, x, y, p->eta_d.as<double>(), 1.0, nullptr,
                                      0.0, as_stream(stream));
    });
}

sip_status sip_apply_A_f32(sip_problem* p, const float* x, float* y, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded(p->ctx, [&] {
        sip::require(x && y, "null vector");
        sip::require(x != y, "x and y must not overlap");
        sip::launch_apply_sip<float>(p->n, p->geom, x, y, p->eta_f.as<float>(), 1.0f, nullptr,
                                     0.0f, as_stream(stream));
    });
}

sip_status sip_apply_B(sip_problem* p, const double* xp, double* yu, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded(p->ctx, [&] {
        sip::require(xp && yu, "null vector");
        sip::launch_apply_B<double>(p->k, p->geom, xp, yu, as_stream(stream));
    });
}

sip_status sip_apply_Bt(sip_problem* p, const double* xu, double* yp, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded(p->ctx, [&] {
        sip::require(xu && yp, "null vector");
        sip::launch_apply_Bt<double>(p->k, p->geom, xu, yp, as_stream(stream));
    });
}

sip_status sip_rasterise_inclusions(sip_ctx* ctx, int nx, int ny, double lx, double ly,
                                    const double* shapes, int n_shapes, double eta_bg,
                                    double rho_bg, double* eta_out, double* rho_out,
                                    void* stream) {
    if (!ctx) return SIP_ERR_INVALID_ARG;
    return guarded(ctx, [&] {
        sip::require(nx >= 1 && ny >= 1 && std::isfinite(lx) && std::isfinite(ly) && lx > 0 &&
                         ly > 0,
                     "bad mesh");
        sip::require(n_shapes >= 0 && (n_shapes == 0 || shapes), "bad inclusion list");
        sip::require(eta_out && rho_out, "null output");
        sip::require(std::isfinite(eta_bg) && eta_bg > 0 && std::isfinite(rho_bg),
                     "bad background material");
        for (int i = 0; i < n_shapes; ++i) {
            const double* s = shapes + 7 * i;
            for (int j = 0; j < 7; ++j)
                sip::require(std::isfinite(s[j]), "non-finite inclusion record");
            sip::require(s[0] == 0.0 || s[0] == 1.0, "unknown inclusion kind");
            sip::require(s[0] != 0.0 || s[3] >= 0, "negative radius");
            sip::require(s[5] >= eta_bg && s[6] >= rho_bg,
                         "inclusions must be at least as viscous and dense as the background");
        }
        SIP_CUDA(cudaSetDevice(ctx->device));
        sip::DeviceBuffer d;
        if (n_shapes > 0) {
            d.alloc(size_t(n_shapes) * 7 * sizeof(double));
            SIP_CUDA(cudaMemcpyAsync(d.ptr, shapes, size_t(n_shapes) * 7 * sizeof(double),
                                     cudaMemcpyHostToDevice, as_stream(stream)));
        }
        sip::launch_rasterise(nx, ny, lx, ly, d.as<double>(), n_shapes, eta_bg, rho_bg, eta_out,
                              rho_out, as_stream(stream));
        SIP_CUDA(cudaStreamSynchronize(as_stream(stream)));   // d is freed on return
    });
}

sip_status sip_rhs_body_force(sip_problem* p, const double* rho, double g, double* f,
                              void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded(p->ctx, [&] {
        sip::require(rho && f, "null vector");
        sip::require(std::isfinite(g), "non-finite gravity");
        sip::launch_rhs_body_force(p->k, p->geom, rho, g, f, as_stream(stream));
    });
}

}  // extern "C"
