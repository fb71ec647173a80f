// extern "C" entry points of the SIP-DG Stokes library: argument checks,
// error translation, and dispatch to the kernels.  No C++ exception leaves
// this file.
#include <cstring>

#include "sip_solver.h"

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

// guarded() with the library's allocations ordered on the caller's stream
template <typename F>
sip_status guarded_s(sip_ctx* ctx, void* stream, F&& f) {
    sip::AllocStreamScope scope(as_stream(stream));
    return guarded(ctx, std::forward<F>(f));
}


}  // namespace


namespace sip {

void require_valid_opts(const sip_solve_opts& o, int precision) {
    require(std::isfinite(o.rtol) && o.rtol > 0 && o.max_outer >= 1 && o.restart >= 1 &&
                o.restart <= 250 && std::isfinite(o.inner_rtol) && o.inner_rtol > 0 &&
                o.max_inner >= 1 && (o.inner_loop == 0 || o.inner_loop == 1) &&
                o.inner_krylov >= 0 && o.inner_krylov <= 3 &&
                !(o.inner_loop == 1 && o.inner_krylov >= 2) &&
                (o.inner_norm == 0 || o.inner_norm == 1) &&
                !(o.inner_loop == 1 && o.inner_norm == 1),
            "bad solve options");
    require(o.inner_krylov != 3 || (o.inner_restart >= 1 && o.inner_restart <= 64 &&
                                    precision != SIP_PREC_MIXED_F32_INNER),
            "GCR needs 1 <= inner_restart <= 64 and an FP64 inner iterate");
    require(o.outer_krylov == 0 || o.outer_krylov == 1, "outer_krylov is 0 or 1");
    require(o.refine >= 0 && o.refine <= 100, "refine is 0..100");
    require(std::isfinite(o.time_limit_ms) && o.time_limit_ms >= 0.0,
            "time_limit_ms must be finite and >= 0");
}

const char* status_message(sip_status st) {
    switch (st) {
        case SIP_ERR_NOT_CONVERGED: return "the solve did not reach the tolerance";
        case SIP_ERR_BREAKDOWN: return "Krylov breakdown";
        case SIP_ERR_TIMEOUT: return "the solve passed its time limit";
        case SIP_ERR_CANCELLED: return "the solve was cancelled";
        default: return "the solve failed";
    }
}

}  // namespace sip

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
    d->coarse = SIP_COARSE_Q1;
    d->cheb_steps_p = 2;
    d->cheb_steps_h = 3;
    d->eig_iters = 10;
    d->cheb_lo = 0.1;
    d->cheb_hi = 1.1;
    d->seed = 0;
    d->precision = SIP_PREC_FP64;
    d->mixed_fp64_ratio = 1e3;
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
        sip::require(d->precision >= SIP_PREC_FP64 && d->precision <= SIP_PREC_MIXED_F32_INNER,
                     "unknown precision");
        sip::require(d->cheb_steps_p >= 1 && d->cheb_steps_h >= 1 && d->eig_iters >= 1 &&
                         d->eig_iters <= 100,
                     "smoothing steps and eigen-estimate iterations must be positive (<= 100)");
        sip::require(std::isfinite(d->cheb_lo) && std::isfinite(d->cheb_hi) && d->cheb_lo > 0 &&
                         d->cheb_hi > d->cheb_lo,
                     "Chebyshev bound factors must satisfy 0 < lo < hi");
        sip::require(std::isfinite(d->mixed_fp64_ratio) && d->mixed_fp64_ratio >= 0.0,
                     "mixed_fp64_ratio must be finite and >= 0");
        sip::require(d->coarse == SIP_COARSE_Q1 || d->coarse == SIP_COARSE_Q0,
                     "unknown coarse space");
        {
            // Q^2_1: the mesh vertices are coarsened; Q^2_0: the element
            // centres, an (nx-1) x (ny-1) grid of intervals
            int cx = d->coarse == SIP_COARSE_Q0 ? d->nx - 1 : d->nx;
            int cy = d->coarse == SIP_COARSE_Q0 ? d->ny - 1 : d->ny;
            for (int l = 0; l < d->n_hlevels; ++l) {
                sip::require(cx % 2 == 0 && cy % 2 == 0 && cx > 0 && cy > 0,
                             "mesh cannot be coarsened n_hlevels times");
                cx /= 2;
                cy /= 2;
            }
        }
        if (d->coarse == SIP_COARSE_Q0 && d->n_hlevels == 0)
            sip::require(int64_t(d->nx) * d->ny <= 8192,
                         "A_p(Q^2_0) coarse direct solve limited to 8192 elements; use n_hlevels > 0");
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
            const cudaStream_t s = sip::alloc_stream();
            p->eta_d.alloc(ne * sizeof(double));
            SIP_CUDA(cudaMemcpyAsync(p->eta_d.ptr, eta.data(), ne * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
            p->derive_eta(s);
            SIP_CUDA(cudaStreamSynchronize(s));
        } catch (...) {
            delete p;
            throw;
        }
        *out = p;
    });
}

void sip_problem_destroy(sip_problem* p) {
    if (!p) return;
    // the problem's buffers may still be in use on any stream the caller
    // used: wait for the device before returning them to the pool
    cudaSetDevice(p->ctx->device);
    cudaDeviceSynchronize();
    sip::ReleaseOnLegacyScope legacy;   // its allocation streams may be destroyed by now
    delete p;
}

sip_status sip_problem_sizes(const sip_problem* p, int64_t* n_u, int64_t* n_p,
                             int64_t* device_bytes) {
    if (!p) return SIP_ERR_INVALID_ARG;
    if (n_u) *n_u = p->n_u;
    if (n_p) *n_p = p->n_p;
    if (device_bytes) *device_bytes = p->device_bytes();
    return SIP_OK;
}

sip_status sip_problem_schedule(const sip_problem* p, int apply[2], int fused[2]) {
    if (!p) return SIP_ERR_INVALID_ARG;
    for (int t = 0; t < 2; ++t) {
        if (apply) {
            const int v = p->geom.variant[t];
            apply[t] = v != sip::APPLY_AUTO ? v : (p->n <= 6 ? int(sip::APPLY_ELEM2)
                                                             : int(sip::APPLY_TILE));
            if (apply[t] == int(sip::APPLY_STAGE) && p->geom.stage_rows[t] == 4) apply[t] = 5;
            if (t == 1 && p->geom.n_hi > 0 && p->n <= 6) apply[t] = int(sip::APPLY_STAGE);
        }
        if (fused) fused[t] = (p->n <= 4 && p->geom.fused[t]) ? 1 : 0;
    }
    return SIP_OK;
}

sip_status sip_problem_set_schedule(sip_problem* p, const int apply[2], const int fused[2]) {
    if (!p) return SIP_ERR_INVALID_ARG;
    for (int t = 0; t < 2; ++t) {
        if (apply && (apply[t] < 0 || apply[t] > 6 || (apply[t] != 0 && apply[t] != 3 && p->n > 6) ||
                      (apply[t] == 6 && t == 0))) {
            p->ctx->err = "schedule: apply code outside 0..6, an element kernel above k = 5, or "
                          "code 6 for the FP64 operator";
            return SIP_ERR_INVALID_ARG;
        }
        if (fused && (fused[t] < -1 || fused[t] > 1)) {
            p->ctx->err = "schedule: fused code outside -1..1";
            return SIP_ERR_INVALID_ARG;
        }
    }
    for (int t = 0; t < 2; ++t) {
        if (apply) {
            p->pin_apply[t] = apply[t];
            if (apply[t] > 0) {
                p->geom.variant[t] = apply[t] == 5 ? int(sip::APPLY_STAGE) : apply[t];
                p->geom.stage_rows[t] = apply[t] == 5 ? 4 : 2;
            }
        }
        if (fused) {
            p->pin_fused[t] = fused[t];
            if (fused[t] >= 0) p->geom.fused[t] = fused[t];
        }
    }
    // the captured V-cycles hold the old kernels: rebuild at the next use
    if (p->mg64) p->mg64->ready = false;
    if (p->mg32) p->mg32->ready = false;
    return SIP_OK;
}

sip_status sip_problem_update_eta(sip_problem* p, const double* eta, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(eta != nullptr, "null eta");
        cudaPointerAttributes at{};
        SIP_CUDA(cudaPointerGetAttributes(&at, eta));
        const bool on_dev = at.type == cudaMemoryTypeDevice || at.type == cudaMemoryTypeManaged;
        const cudaStream_t s = as_stream(stream);
        const size_t ne = size_t(p->ne);
        if (on_dev) {
            SIP_CUDA(cudaMemcpyAsync(p->eta_d.ptr, eta, ne * sizeof(double),
                                     cudaMemcpyDeviceToDevice, s));
        } else {
            for (size_t e = 0; e < ne; ++e)
                sip::require(std::isfinite(eta[e]) && eta[e] > 0.0,
                             "eta must be finite and positive");
            SIP_CUDA(cudaMemcpyAsync(p->eta_d.ptr, eta, ne * sizeof(double),
                                     cudaMemcpyHostToDevice, s));
        }
        if (on_dev && !sip::eta_valid(ne, p->eta_d.as<double>(), s))
            throw Error(SIP_ERR_INVALID_ARG, "eta must be finite and positive");
        p->derive_eta(s);
        if (p->mg64) p->mg64->ready = false;
        if (p->mg32) p->mg32->ready = false;
        if (p->ws) p->ws->sinv_ready = false;
    });
}

sip_status sip_apply_A(sip_problem* p, const double* x, double* y, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(x && y, "null vector");
        sip::require(x != y, "x and y must not overlap");
        sip::launch_apply_sip<double>(p->n, p->geom, x, y, p->eta_d.as<double>(), 1.0, nullptr,
                                      0.0, as_stream(stream));
    });
}

sip_status sip_apply_A_f32(sip_problem* p, const float* x, float* y, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(x && y, "null vector");
        sip::require(x != y, "x and y must not overlap");
        sip::launch_apply_sip<float>(p->n, p->geom, x, y, p->eta_f.as<float>(), 1.0f, nullptr,
                                     0.0f, as_stream(stream));
    });
}

sip_status sip_apply_B(sip_problem* p, const double* xp, double* yu, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(xp && yu, "null vector");
        sip::launch_apply_B<double>(p->k, p->geom, xp, yu, as_stream(stream));
    });
}

sip_status sip_apply_Bt(sip_problem* p, const double* xu, double* yp, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(xu && yp, "null vector");
        sip::launch_apply_Bt<double>(p->k, p->geom, xu, yp, as_stream(stream));
    });
}

sip_status sip_rasterise_inclusions(sip_ctx* ctx, int nx, int ny, double lx, double ly,
                                    const double* shapes, int n_shapes, double eta_bg,
                                    double rho_bg, double* eta_out, double* rho_out,
                                    void* stream) {
    if (!ctx) return SIP_ERR_INVALID_ARG;
    return guarded_s(ctx, stream, [&] {
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
    return guarded_s(p->ctx, stream, [&] {
        sip::require(rho && f, "null vector");
        sip::require(std::isfinite(g), "non-finite gravity");
        sip::launch_rhs_body_force(p->k, p->geom, rho, g, f, as_stream(stream));
    });
}

// ------------------------------------------------------------ multigrid
namespace {

sip::Multigrid<double>& mg64(sip_problem* p, cudaStream_t s) {
    SIP_CUDA(cudaSetDevice(p->ctx->device));
    if (!p->mg64) {
        p->mg64 = std::make_unique<sip::Multigrid<double>>();
        p->mg64->P = p;
    }
    if (!p->mg64->ready) p->mg64->setup(s);
    return *p->mg64;
}

sip::Multigrid<float>& mg32(sip_problem* p, cudaStream_t s) {
    SIP_CUDA(cudaSetDevice(p->ctx->device));
    if (!p->mg32) {
        p->mg32 = std::make_unique<sip::Multigrid<float>>();
        p->mg32->P = p;
    }
    if (!p->mg32->ready) p->mg32->setup(s);
    return *p->mg32;
}

}  // namespace

sip_status sip_problem_setup(sip_problem* p, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        SIP_CUDA(cudaSetDevice(p->ctx->device));
        p->ensure_setup(as_stream(stream));
    });
}

sip_status sip_lambda_max(sip_problem* p, int level, double* out) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded(p->ctx, [&] {
        sip::require(out != nullptr, "null output");
        auto& m = mg64(p, nullptr);
        sip::require(level == -1 || (level >= 0 && level < int(m.h.size()) - 1),
                     "level must be -1 (p-level) or a smoothed h-level");
        *out = level < 0 ? m.lmax_p : m.h[level].lmax;
    });
}

sip_status sip_block_jacobi(sip_problem* p, const double* r, double* z, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(r && z && r != z, "bad vectors");
        mg64(p, as_stream(stream)).bj(r, z, as_stream(stream));
    });
}

sip_status sip_p_restrict(sip_problem* p, const double* r, double* r1, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(r && r1, "null vector");
        sip::launch_p_restrict<double>(size_t(p->ne), p->n, r, r1, as_stream(stream));
    });
}

sip_status sip_p_prolong_add(sip_problem* p, const double* e1, double* y, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(e1 && y, "null vector");
        sip::launch_p_prolong_add<double>(size_t(p->ne), p->n, e1, y, as_stream(stream));
    });
}

sip_status sip_apply_A1(sip_problem* p, const double* x1, double* y1, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(x1 && y1 && x1 != y1, "bad vectors");
        sip::launch_apply_sip<double>(2, p->geom1, x1, y1, p->eta_d.as<double>(), 1.0, nullptr, 0.0,
                                      as_stream(stream));
    });
}

sip_status sip_cd_prolong(sip_problem* p, const double* v, double* u1, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(v && u1, "null vector");
        sip::launch_pcd<double>(p->desc.nx, p->desc.ny, v, u1, as_stream(stream));
    });
}

sip_status sip_dc_restrict(sip_problem* p, const double* u1, double* v, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(v && u1, "null vector");
        sip::launch_rdc<double>(p->desc.nx, p->desc.ny, u1, v, as_stream(stream));
    });
}

sip_status sip_hlevel_dims(sip_problem* p, int level, int* n_levels, int* nvx, int* nvy) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded(p->ctx, [&] {
        auto& m = mg64(p, nullptr);
        if (n_levels) *n_levels = int(m.h.size());
        if (level >= 0) {
            sip::require(level < int(m.h.size()), "no such level");
            if (nvx) *nvx = m.h[level].nvx;
            if (nvy) *nvy = m.h[level].nvy;
        }
    });
}

sip_status sip_hlevel_stencil(sip_problem* p, int level, double* S, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        auto& m = mg64(p, as_stream(stream));
        sip::require(S != nullptr, "null output");
        sip::require(level >= 0 && level < int(m.h.size()), "no such level");
        SIP_CUDA(cudaMemcpyAsync(S, m.h[level].S.ptr, m.h[level].S.bytes, cudaMemcpyDeviceToDevice,
                                 as_stream(stream)));
    });
}

sip_status sip_hlevel_apply(sip_problem* p, int level, const double* x, double* y, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        auto& m = mg64(p, as_stream(stream));
        sip::require(x && y && x != y, "bad vectors");
        sip::require(level >= 0 && level < int(m.h.size()), "no such level");
        m.hlevel_apply(level, x, y, as_stream(stream));
    });
}

sip_status sip_coarse_solve(sip_problem* p, const double* b, double* x, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        auto& m = mg64(p, as_stream(stream));
        sip::require(b && x && b != x, "bad vectors");
        sip::launch_dense_symv<double>(m.nc, m.cinv.as<double>(), b, x, as_stream(stream));
    });
}

sip_status sip_vcycle(sip_problem* p, const double* r, double* z, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(r && z && r != z, "bad vectors");
        mg64(p, as_stream(stream)).vcycle(r, z, as_stream(stream));
    });
}

sip_status sip_vcycle_f32(sip_problem* p, const float* r, float* z, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(r && z && r != z, "bad vectors");
        mg32(p, as_stream(stream)).vcycle(r, z, as_stream(stream));
    });
}

sip_status sip_inner_solve(sip_problem* p, const double* t, double* y, double rtol, int max_it,
                           int* its, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(t && y && t != y, "bad vectors");
        sip::require(rtol > 0 && max_it >= 1, "bad tolerance or iteration cap");
        const int n = mg64(p, as_stream(stream)).inner_pcg(t, y, rtol, max_it, as_stream(stream),
                                                          nullptr);
        SIP_CUDA(cudaStreamSynchronize(as_stream(stream)));
        if (its) *its = n;
    });
}

void sip_solve_opts_default(sip_solve_opts* o) {
    if (!o) return;
    o->rtol = 1e-8;
    o->max_outer = 500;
    o->restart = 100;
    o->inner_rtol = 1e-3;
    o->max_inner = 200;
    o->inner_loop = 0;
    o->inner_krylov = 0;
    o->inner_norm = 0;
    o->inner_restart = 30;
    o->outer_krylov = 0;
    o->refine = 0;
    o->time_limit_ms = 0.0;
}

sip_status sip_residual_dd(sip_problem* p, const double* f, const double* g, const double* x_u,
                           const double* x_p, double* r_u, double* r_p, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    return guarded_s(p->ctx, stream, [&] {
        sip::require(f && x_u && x_p && r_u && r_p, "null vector");
        sip::require(r_u != x_u && r_p != x_p && r_u != x_p && r_p != x_u,
                     "r and x must not overlap");
        SIP_CUDA(cudaSetDevice(p->ctx->device));
        sip::residual_dd(p, f, g, x_u, x_p, r_u, r_p, as_stream(stream));
    });
}

sip_status sip_solve_dd(sip_problem* p, const double* f, const double* g, double* u_dd,
                        double* p_dd, const sip_solve_opts* opts, sip_solve_report* rep,
                        void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    sip_status st = SIP_OK;
    const sip_status gst = guarded(p->ctx, [&] {
        sip::require(f && u_dd && p_dd, "null vector");
        sip::require(opts && opts->refine > 0, "sip_solve_dd needs opts->refine > 0");
        const sip_solve_opts o = *opts;
        sip::require_valid_opts(o, p->desc.precision);
        SIP_CUDA(cudaSetDevice(p->ctx->device));
        const sip::StopScope stop(o.time_limit_ms > 0.0 ? sip::steady_ms() + o.time_limit_ms : 0.0,
                                  nullptr);
        st = sip::run_solve_refined(p, f, g, nullptr, nullptr, o, rep, as_stream(stream), u_dd,
                                    p_dd);
        if (st != SIP_OK) throw Error(st, sip::status_message(st));
    });
    if (gst != SIP_OK && rep) rep->status = gst;
    return gst;
}

sip_status sip_solve(sip_problem* p, const double* f, const double* g, double* u, double* pp,
                     const sip_solve_opts* opts, sip_solve_report* rep, void* stream) {
    if (!p) return SIP_ERR_INVALID_ARG;
    sip_status st = SIP_OK;
    const sip_status gst = guarded(p->ctx, [&] {
        sip::require(f && u && pp, "null vector");
        sip_solve_opts o;
        sip_solve_opts_default(&o);
        if (opts) o = *opts;
        sip::require_valid_opts(o, p->desc.precision);
        SIP_CUDA(cudaSetDevice(p->ctx->device));
        const sip::StopScope stop(o.time_limit_ms > 0.0 ? sip::steady_ms() + o.time_limit_ms : 0.0,
                                  nullptr);
        st = sip::solve_dispatch(p, f, g, u, pp, o, rep, as_stream(stream));
        if (st != SIP_OK) throw Error(st, sip::status_message(st));
    });
    if (gst != SIP_OK && rep) rep->status = gst;
    return gst;
}

}  // extern "C"
