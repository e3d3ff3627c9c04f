// The C ABI of include/ccov.h: host-side validation, index construction,
// device memory and the order of the kernel launches of steps (a)-(d).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <new>
#include <vector>

#include "ccov_internal.cuh"
#include "../../include/ccov_surrogate.h"

using ccov::Ctx;

struct ccov_ctx {
    Ctx c;
};

namespace {

ccov_status fail(Ctx* c, ccov_status s, const char* fmt, ...) {
    if (c) {
        char buf[512];
        va_list ap;
        va_start(ap, fmt);
        vsnprintf(buf, sizeof buf, fmt, ap);
        va_end(ap);
        c->err = buf;
    }
    return s;
}

ccov_status cuda_fail(Ctx* c, cudaError_t e, const char* where) {
    if (e == cudaErrorMemoryAllocation)
        return fail(c, CCOV_ERR_OOM, "%s: %s", where, cudaGetErrorString(e));
    return fail(c, CCOV_ERR_CUDA, "%s: %s", where, cudaGetErrorString(e));
}

#define CK(expr, where)                                   \
    do {                                                  \
        cudaError_t _e = (expr);                          \
        if (_e != cudaSuccess) return cuda_fail(&c, _e, where); \
    } while (0)

template <class T>
cudaError_t dalloc(Ctx& c, T** p, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), count * sizeof(T));
    if (e == cudaSuccess) c.bytes += (int64_t)(count * sizeof(T));
    return e;
}

void free_all(Ctx& c) {
    void* ptrs[] = {c.d_cams, c.d_pts, c.d_obs, c.d_obscov, c.d_pt_ptr, c.d_cam_ptr, c.d_cam_perm,
                    c.d_camprep, c.d_W, c.d_Ainv, c.d_U, c.d_Z, c.d_Gp, c.d_W7, c.d_HP, c.d_R,
                    c.d_P, c.d_Linv, c.d_F, c.d_G, c.d_D, c.d_Sig, c.d_small, c.d_flag,
                    c.d_V, c.d_J, c.d_pair_desc, c.d_pair_ent, c.d_w7part, c.d_sgauge};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    ccov::mixed_free(c);
    ccov::est_free(c);
    ccov::update_free(c);
    for (auto& e : c.ev)
        if (e) cudaEventDestroy(e);
    for (auto& e : c.prof_ev)
        if (e) cudaEventDestroy(e);
    if (c.own_stream && c.stream) cudaStreamDestroy(c.stream);
}

bool finite_all(const double* p, int64_t k) {
    for (int64_t i = 0; i < k; ++i)
        if (!std::isfinite(p[i])) return false;
    return true;
}

// Host validation of the scene and construction of the two indices:
// pt_ptr (CSR by point over the point-sorted observations) and the camera
// grouping cam_ptr / cam_perm (counting sort by camera).
ccov_status build_index(Ctx& c, const double* cams, const double* pts, const ccov_obs* obs,
                        const double* cov, std::vector<int>& pt_ptr, std::vector<int>& cam_ptr,
                        std::vector<int>& cam_perm) {
    const int64_t n = c.n, m = c.m, t = c.t;
    if (!finite_all(cams, 9 * n)) return fail(&c, CCOV_ERR_INVALID_ARG, "non-finite camera parameter");
    if (!finite_all(pts, 3 * m)) return fail(&c, CCOV_ERR_INVALID_ARG, "non-finite point");
    pt_ptr.assign(m + 1, 0);
    cam_ptr.assign(n + 1, 0);
    std::vector<int64_t> stamp(n, -1);
    int64_t prev = -1;
    for (int64_t o = 0; o < t; ++o) {
        const ccov_obs& r = obs[o];
        if (r.cam < 0 || r.cam >= n || r.pt < 0 || r.pt >= m)
            return fail(&c, CCOV_ERR_INVALID_ARG, "observation %lld: index out of range", (long long)o);
        if (r.pt < prev)
            return fail(&c, CCOV_ERR_INVALID_ARG, "observations must be sorted by point (at %lld)", (long long)o);
        if (!std::isfinite(r.u[0]) || !std::isfinite(r.u[1]))
            return fail(&c, CCOV_ERR_INVALID_ARG, "observation %lld: non-finite u", (long long)o);
        if (stamp[r.cam] == r.pt)
            return fail(&c, CCOV_ERR_INVALID_ARG, "point %d observed twice by camera %d", r.pt, r.cam);
        stamp[r.cam] = r.pt;
        prev = r.pt;
        pt_ptr[r.pt + 1]++;
        cam_ptr[r.cam + 1]++;
        if (cov) {
            const double* s = cov + 4 * o;
            if (!finite_all(s, 4) || !(s[0] > 0.0) || !(s[0] * s[3] - s[1] * s[2] > 0.0) ||
                std::fabs(s[1] - s[2]) > 1e-12 * (std::fabs(s[1]) + std::fabs(s[2]) + 1e-300))
                return fail(&c, CCOV_ERR_INVALID_ARG, "observation %lld: covariance not SPD", (long long)o);
        }
    }
    for (int64_t j = 0; j < m; ++j) {
        if (pt_ptr[j + 1] < 2)
            return fail(&c, CCOV_ERR_DEGENERATE, "point %lld has %d observations (< 2)", (long long)j, pt_ptr[j + 1]);
        pt_ptr[j + 1] += pt_ptr[j];
    }
    for (int64_t i = 0; i < n; ++i) {
        if (cam_ptr[i + 1] < 2)
            return fail(&c, CCOV_ERR_DEGENERATE, "camera %lld has %d observations (< 2)", (long long)i, cam_ptr[i + 1]);
        cam_ptr[i + 1] += cam_ptr[i];
    }
    cam_perm.resize(t);
    std::vector<int> fill(cam_ptr.begin(), cam_ptr.end() - 1);
    for (int64_t o = 0; o < t; ++o) cam_perm[fill[obs[o].cam]++] = (int)o;
    return CCOV_OK;
}

// The blocks Z_ik (i >= k) that receive Schur terms and, per block, the
// observation pairs of the points that cameras i and k share (Eq.
// schur-complement-inversion: Z_ik = [i = k] U_i - sum_j W_ij A_j^-1 W_kj^T).
// The entries are ordered by block (row i, then column k; two stable
// counting sorts) and within a block by point, so the device sums every block
// in a fixed order.  Depends on S only (ccov_load keeps it).
void build_pairs(const ccov_obs* obs, int64_t n, int64_t m, const std::vector<int>& pt_ptr,
                 std::vector<int4>& desc, std::vector<int2>& ent, const std::vector<char>& fixed) {
    int64_t total = 0;
    for (int64_t j = 0; j < m; ++j) {
        if (!fixed.empty() && fixed[j]) continue;
        const int64_t L = pt_ptr[j + 1] - pt_ptr[j];
        total += L * (L + 1) / 2;
    }
    std::vector<int> row(total), col(total);
    std::vector<int2> raw(total);
    int64_t e = 0;
    for (int64_t j = 0; j < m; ++j) {
        if (!fixed.empty() && fixed[j]) continue;   // a fixed point is not eliminated (Alg. 5)
        for (int a = pt_ptr[j]; a < pt_ptr[j + 1]; ++a)
            for (int b = a; b < pt_ptr[j + 1]; ++b) {
                const int ca = obs[a].cam, cb = obs[b].cam;
                const bool first = ca >= cb;
                row[e] = first ? ca : cb;
                col[e] = first ? cb : ca;
                raw[e] = make_int2(first ? a : b, first ? b : a);
                ++e;
            }
    }
    // stable counting sort by column, then by row: (row, col, point) order
    std::vector<int64_t> cnt(n + 1);
    std::vector<int64_t> by_col(total), order(total);
    for (int64_t q = 0; q < total; ++q) cnt[col[q] + 1]++;
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    for (int64_t q = 0; q < total; ++q) by_col[cnt[col[q]]++] = q;
    std::fill(cnt.begin(), cnt.end(), 0);
    for (int64_t q = 0; q < total; ++q) cnt[row[q] + 1]++;
    for (int64_t i = 0; i < n; ++i) cnt[i + 1] += cnt[i];
    for (int64_t q : by_col) order[cnt[row[q]]++] = q;
    ent.resize(total);
    desc.clear();
    for (int64_t q = 0; q < total; ++q) {
        const int64_t src = order[q];
        ent[q] = raw[src];
        if (q == 0 || row[src] != row[order[q - 1]] || col[src] != col[order[q - 1]])
            desc.push_back(make_int4(row[src], col[src], (int)q, 0));
        desc.back().w++;
    }
}

// The three fixed points of Alg. 5 when the caller gives none: the point
// farthest from the centroid, the point farthest from it, the point
// farthest from the line through those two (ties: the smaller index).
void three_far_points(const double* pts, int64_t m, int out[3]) {
    double c[3] = {0, 0, 0};
    for (int64_t j = 0; j < m; ++j)
        for (int a = 0; a < 3; ++a) c[a] += pts[3 * j + a];
    for (int a = 0; a < 3; ++a) c[a] /= (double)m;
    auto far_from = [&](const double* q) {
        int64_t best = 0;
        double bd = -1.0;
        for (int64_t j = 0; j < m; ++j) {
            double d = 0.0;
            for (int a = 0; a < 3; ++a) d += (pts[3 * j + a] - q[a]) * (pts[3 * j + a] - q[a]);
            d = std::sqrt(d);
            if (d > bd) { bd = d; best = j; }
        }
        return best;
    };
    const int64_t p1 = far_from(c), p2 = far_from(pts + 3 * p1);
    double u[3], nu = 0.0;
    for (int a = 0; a < 3; ++a) { u[a] = pts[3 * p2 + a] - pts[3 * p1 + a]; nu += u[a] * u[a]; }
    nu = std::sqrt(nu);
    for (int a = 0; a < 3; ++a) u[a] /= nu;
    int64_t p3 = 0;
    double bd = -1.0;
    for (int64_t j = 0; j < m; ++j) {
        double v[3], vu = 0.0, d = 0.0;
        for (int a = 0; a < 3; ++a) { v[a] = pts[3 * j + a] - pts[3 * p1 + a]; vu += v[a] * u[a]; }
        for (int a = 0; a < 3; ++a) d += (v[a] - vu * u[a]) * (v[a] - vu * u[a]);
        d = std::sqrt(d);
        if (d > bd) { bd = d; p3 = j; }
    }
    out[0] = (int)p1; out[1] = (int)p2; out[2] = (int)p3;
}

ccov_status check_device(Ctx& c, const char* where) {
    cudaError_t e = cudaStreamSynchronize(c.stream);
    if (e != cudaSuccess) return cuda_fail(&c, e, where);
    int flag[2] = {0, 0};
    e = cudaMemcpy(flag, c.d_flag, sizeof flag, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(&c, e, where);
    switch (flag[0]) {
        case ccov::DEV_OK: return CCOV_OK;
        case ccov::DEV_BEHIND:
            return fail(&c, CCOV_ERR_DEGENERATE, "%s: point behind camera (observation %d)", where, flag[1]);
        case ccov::DEV_SINGULAR_A:
            return fail(&c, CCOV_ERR_DEGENERATE, "%s: point block A_j singular (point %d)", where, flag[1]);
        case ccov::DEV_NOT_SPD:
            return fail(&c, CCOV_ERR_DEGENERATE, "%s: reduced camera matrix not positive definite (row %d)", where, flag[1]);
        case ccov::DEV_SINGULAR_W7:
            return fail(&c, CCOV_ERR_DEGENERATE, "%s: W7 singular (column %d)", where, flag[1]);
        case ccov::DEV_SINGULAR_JR:
            return fail(&c, CCOV_ERR_DEGENERATE, "%s: J_r^T J_r singular (camera %d)", where, flag[1]);
        case ccov::DEV_TIMEOUT:
            return fail(&c, CCOV_ERR_TIMEOUT, "%s: device wait gave up (site %d)", where, flag[1]);
        case ccov::DEV_SMEM_ALIGN:
            return fail(&c, CCOV_ERR_CUDA, "%s: shared memory window of the GEMM not 1024-byte aligned", where);
        case ccov::DEV_RANGE:
            return fail(&c, CCOV_ERR_NOT_CONVERGED,
                        "%s: the mixed form's fixed-point range was exceeded (row %d): the scene is too "
                        "ill-conditioned for it; use precision FP64", where, flag[1]);
        default:
            return fail(&c, CCOV_ERR_CUDA, "%s: device error code %d", where, flag[0]);
    }
}

float elapsed(Ctx& c, int a, int b) {
    float ms = 0.f;
    cudaEventElapsedTime(&ms, c.ev[a], c.ev[b]);
    return ms;
}

// The centre camera's n x 8 values {r, C, c, k} in the 9-slot layout the
// kernels read (slot 8, no parameter, zero).  `memory` says where src lives.
bool expand_centre(const double* src, int64_t n, int memory, std::vector<double>& out) {
    std::vector<double> tmp(8 * n);
    if (memory == CCOV_MEM_DEVICE) {
        if (cudaMemcpy(tmp.data(), src, sizeof(double) * 8 * n, cudaMemcpyDeviceToHost) != cudaSuccess) return false;
    } else {
        std::memcpy(tmp.data(), src, sizeof(double) * 8 * n);
    }
    out.assign(9 * n, 0.0);
    for (int64_t i = 0; i < n; ++i)
        for (int k = 0; k < 8; ++k) out[9 * i + k] = tmp[8 * i + k];
    return true;
}

ccov_status upload(Ctx& c, const double* cams, const double* pts, const ccov_obs* obs,
                   const double* cov, int memory) {
    cudaMemcpyKind kind = memory == CCOV_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyHostToDevice;
    if (c.opt.camera_model == CCOV_CAMERA_CENTRE8) {
        std::vector<double> e;
        if (!expand_centre(cams, c.n, memory, e)) return fail(&c, CCOV_ERR_INVALID_ARG, "cameras not readable");
        // synchronous: the host vector goes out of scope
        CK(cudaMemcpy(c.d_cams, e.data(), sizeof(double) * 9 * c.n, cudaMemcpyHostToDevice), "copy cameras");
    } else {
        CK(cudaMemcpyAsync(c.d_cams, cams, sizeof(double) * 9 * c.n, kind, c.stream), "copy cameras");
    }
    CK(cudaMemcpyAsync(c.d_pts, pts, sizeof(double) * 3 * c.m, kind, c.stream), "copy points");
    CK(cudaMemcpyAsync(c.d_obs, obs, sizeof(ccov_obs) * c.t, kind, c.stream), "copy observations");
    if (cov) CK(cudaMemcpyAsync(c.d_obscov, cov, sizeof(double) * 4 * c.t, kind, c.stream), "copy obs_cov");
    return CCOV_OK;
}

}  // namespace

namespace ccov {
ccov_status device_status(Ctx& c, const char* where) { return check_device(c, where); }

void prof_begin(Ctx& c) {
    if (!c.opt.profile || c.capturing) return;
    while (c.prof_ev.size() < c.prof_used + 2) {
        cudaEvent_t e;
        if (cudaEventCreate(&e) != cudaSuccess) return;
        c.prof_ev.push_back(e);
    }
    cudaEventRecord(c.prof_ev[c.prof_used], c.stream);
}
void prof_end(Ctx& c, double flops) {
    if (!c.opt.profile || c.capturing || c.prof_ev.size() < c.prof_used + 2) return;
    cudaEventRecord(c.prof_ev[c.prof_used + 1], c.stream);
    c.prof_used += 2;
    c.prof_flops += flops;
}
}  // namespace ccov

extern "C" {

const char* ccov_status_string(ccov_status s) {
    switch (s) {
        case CCOV_OK: return "ok";
        case CCOV_ERR_INVALID_ARG: return "invalid argument";
        case CCOV_ERR_DEGENERATE: return "degenerate input";
        case CCOV_ERR_NOT_CONVERGED: return "not converged";
        case CCOV_ERR_TIMEOUT: return "device wait timed out";
        case CCOV_ERR_OOM: return "out of device memory";
        case CCOV_ERR_CUDA: return "CUDA error";
    }
    return "unknown status";
}

const char* ccov_last_error(const ccov_ctx* ctx) { return ctx ? ctx->c.err.c_str() : ""; }

ccov_status ccov_create(const double* cameras, int64_t n, const double* points, int64_t m,
                        const ccov_obs* obs, int64_t t, double sigma, const double* obs_cov,
                        const ccov_options* opt, void* stream, ccov_ctx** out) {
    if (!out) return CCOV_ERR_INVALID_ARG;
    *out = nullptr;
    if (!cameras || !points || !obs || n < 1 || m < 3 || t < 4 || t >= (int64_t)1 << 31 ||
        9 * n >= ((int64_t)1 << 31) / 9)
        return CCOV_ERR_INVALID_ARG;
    if (!obs_cov && !(sigma > 0.0 && std::isfinite(sigma))) return CCOV_ERR_INVALID_ARG;
    ccov_ctx* h = new (std::nothrow) ccov_ctx();
    if (!h) return CCOV_ERR_OOM;
    Ctx& c = h->c;
    *out = h;
    if (opt) c.opt = *opt;
    // the comparison algorithms' matrices (Z restricted to its range, or with
    // three points fixed) and the centre camera's are about 100x worse
    // conditioned after Jacobi scaling (2e6 against 2e4): six digits
    if (c.opt.mixed_slices == 0)
        c.opt.mixed_slices = c.opt.gauge == CCOV_GAUGE_NATURAL && c.opt.camera_model == CCOV_CAMERA_RT9 ? 5 : 6;
    if (c.opt.precision != CCOV_PREC_FP64 && c.opt.precision != CCOV_PREC_MIXED)
        return fail(&c, CCOV_ERR_INVALID_ARG, "unknown precision %d", c.opt.precision);
    if (c.opt.mixed_slices < 4 || c.opt.mixed_slices > 6)
        return fail(&c, CCOV_ERR_INVALID_ARG, "mixed_slices must be 4..6");
    if (c.opt.est_cameras == 0) c.opt.est_cameras = ccov::kEstDefaultCams;
    if (c.opt.est_cameras < 1 || c.opt.est_cameras > ccov::kEstMaxCams)
        return fail(&c, CCOV_ERR_INVALID_ARG, "est_cameras must be 1..%d", ccov::kEstMaxCams);
    if (c.opt.nullspace_route != CCOV_NULL_PAPER && c.opt.nullspace_route != CCOV_NULL_CLOSED)
        return fail(&c, CCOV_ERR_INVALID_ARG, "unknown nullspace route");
    if (c.opt.gauge != CCOV_GAUGE_NATURAL && c.opt.gauge != CCOV_GAUGE_ZPINV && c.opt.gauge != CCOV_GAUGE_FIXED3)
        return fail(&c, CCOV_ERR_INVALID_ARG, "unknown gauge");
    if (c.opt.camera_model != CCOV_CAMERA_RT9 && c.opt.camera_model != CCOV_CAMERA_CENTRE8)
        return fail(&c, CCOV_ERR_INVALID_ARG, "unknown camera model");
    c.n = n; c.m = m; c.t = t; c.N = 9 * n;
    c.Np = (c.N + ccov::kNB - 1) / ccov::kNB * ccov::kNB;
    c.sigma = sigma;
    c.has_cov = obs_cov != nullptr;
    c.stats.n = n; c.stats.m = m; c.stats.t = t; c.stats.N = c.N; c.stats.N_pad = c.Np;

    // host copies for validation when the inputs live on the device
    const bool dev = c.opt.input_memory == CCOV_MEM_DEVICE;
    std::vector<double> hc, hp, hcov;
    std::vector<ccov_obs> ho;
    const double* vc = cameras; const double* vp = points; const ccov_obs* vo = obs;
    const double* vcov = obs_cov;
    std::vector<double> hc9;
    if (c.opt.camera_model == CCOV_CAMERA_CENTRE8) {
        if (!expand_centre(cameras, n, dev ? CCOV_MEM_DEVICE : CCOV_MEM_HOST, hc9))
            return fail(&c, CCOV_ERR_INVALID_ARG, "cameras not readable");
        vc = hc9.data();
    }
    if (dev) {
        hc.resize(9 * n); hp.resize(3 * m); ho.resize(t);
        if ((c.opt.camera_model != CCOV_CAMERA_CENTRE8 &&
             cudaMemcpy(hc.data(), cameras, 8 * 9 * n, cudaMemcpyDeviceToHost) != cudaSuccess) ||
            cudaMemcpy(hp.data(), points, 8 * 3 * m, cudaMemcpyDeviceToHost) != cudaSuccess ||
            cudaMemcpy(ho.data(), obs, sizeof(ccov_obs) * t, cudaMemcpyDeviceToHost) != cudaSuccess)
            return fail(&c, CCOV_ERR_INVALID_ARG, "input_memory = device but the inputs are not readable device memory");
        if (c.opt.camera_model != CCOV_CAMERA_CENTRE8) vc = hc.data();
        vp = hp.data(); vo = ho.data();
        if (obs_cov) {
            hcov.resize(4 * t);
            if (cudaMemcpy(hcov.data(), obs_cov, 8 * 4 * t, cudaMemcpyDeviceToHost) != cudaSuccess)
                return fail(&c, CCOV_ERR_INVALID_ARG, "obs_cov is not readable device memory");
            vcov = hcov.data();
        }
    }
    std::vector<int> pt_ptr, cam_ptr, cam_perm;
    ccov_status s = build_index(c, vc, vp, vo, vcov, pt_ptr, cam_ptr, cam_perm);
    if (s != CCOV_OK) return s;
    std::vector<char> fixed;
    if (c.opt.gauge == CCOV_GAUGE_FIXED3) {
        int* fp = c.opt.fixed_points;
        const bool given = !(fp[0] == fp[1] && fp[1] == fp[2] && (fp[0] == -1 || fp[0] == 0));
        if (!given) three_far_points(vp, m, fp);
        fixed.assign(m, 0);
        for (int q = 0; q < 3; ++q) {
            if (fp[q] < 0 || fp[q] >= m || fixed[fp[q]])
                return fail(&c, CCOV_ERR_INVALID_ARG, "fixed_points: three distinct point indices needed");
            fixed[fp[q]] = 1;
        }
    }
    std::vector<int4> pair_desc;
    std::vector<int2> pair_ent;
    build_pairs(vo, n, m, pt_ptr, pair_desc, pair_ent, fixed);
    if ((int64_t)pair_ent.size() >= ((int64_t)1 << 31))
        return fail(&c, CCOV_ERR_INVALID_ARG, "too many camera pairs per point (%lld)", (long long)pair_ent.size());
    c.npairs = (int64_t)pair_desc.size();
    c.nent = (int64_t)pair_ent.size();

    if (stream) {
        c.stream = static_cast<cudaStream_t>(stream);
    } else {
        CK(cudaStreamCreateWithFlags(&c.stream, cudaStreamNonBlocking), "stream");
        c.own_stream = true;
    }
    for (auto& e : c.ev) CK(cudaEventCreate(&e), "event");
    CK(ccov::setup_dense64(), "kernel attributes");
    const int64_t Np = c.Np;
    CK(dalloc(c, &c.d_cams, 9 * n), "alloc");
    CK(dalloc(c, &c.d_pts, 3 * m), "alloc");
    CK(dalloc(c, &c.d_obs, t), "alloc");
    if (obs_cov) CK(dalloc(c, &c.d_obscov, 4 * t), "alloc");
    CK(dalloc(c, &c.d_pt_ptr, m + 1), "alloc");
    CK(dalloc(c, &c.d_cam_ptr, n + 1), "alloc");
    CK(dalloc(c, &c.d_cam_perm, t), "alloc");
    CK(dalloc(c, &c.d_camprep, ccov::kCamPrep * n), "alloc");
    CK(dalloc(c, &c.d_W, 27 * t), "alloc");
    CK(dalloc(c, &c.d_Ainv, 6 * m), "alloc");
    CK(dalloc(c, &c.d_U, 45 * n), "alloc");
    CK(dalloc(c, &c.d_Z, Np * Np), "alloc Z");
    CK(dalloc(c, &c.d_V, 27 * t), "alloc");
    CK(dalloc(c, &c.d_J, 24 * t), "alloc");
    CK(dalloc(c, &c.d_pair_desc, c.npairs), "alloc");
    CK(dalloc(c, &c.d_pair_ent, c.nent), "alloc");
    c.w7_wps = ccov::w7_warps_for(m);
    CK(dalloc(c, &c.d_w7part, 56 * (size_t)c.w7_wps), "alloc");
    CK(dalloc(c, &c.d_Gp, 7 * c.N), "alloc");
    CK(dalloc(c, &c.d_W7, 128), "alloc");
    CK(dalloc(c, &c.d_HP, 63 * n), "alloc");
    CK(dalloc(c, &c.d_F, 7 * c.N), "alloc");
    CK(dalloc(c, &c.d_G, 7 * c.N), "alloc");
    CK(dalloc(c, &c.d_D, Np), "alloc");
    CK(dalloc(c, &c.d_Sig, 81 * n), "alloc");
    CK(dalloc(c, &c.d_small, 256), "alloc");
    CK(dalloc(c, &c.d_sgauge, 28 * ccov::kSurrGaugeBlocks + 49), "alloc");
    CK(dalloc(c, &c.d_flag, 2), "alloc");
    CK(dalloc(c, &c.d_Linv, (Np / ccov::kNB) * ccov::kNB * ccov::kNB), "alloc");
    if (c.opt.precision == CCOV_PREC_FP64) {
        CK(dalloc(c, &c.d_R, Np * Np), "alloc R");
        CK(dalloc(c, &c.d_P, Np * ccov::kNB), "alloc");
    } else {
        CK(ccov::mixed_alloc(c), "alloc mixed workspace");
    }
    c.stats.bytes_device = c.bytes;
    CK(cudaMemsetAsync(c.d_flag, 0, 2 * sizeof(int), c.stream), "memset");
    s = upload(c, cameras, points, obs, obs_cov, dev ? CCOV_MEM_DEVICE : CCOV_MEM_HOST);
    if (s != CCOV_OK) return s;
    CK(cudaMemcpyAsync(c.d_pt_ptr, pt_ptr.data(), sizeof(int) * (m + 1), cudaMemcpyHostToDevice, c.stream), "copy");
    CK(cudaMemcpyAsync(c.d_cam_ptr, cam_ptr.data(), sizeof(int) * (n + 1), cudaMemcpyHostToDevice, c.stream), "copy");
    CK(cudaMemcpyAsync(c.d_cam_perm, cam_perm.data(), sizeof(int) * t, cudaMemcpyHostToDevice, c.stream), "copy");
    CK(cudaMemcpyAsync(c.d_pair_desc, pair_desc.data(), sizeof(int4) * c.npairs, cudaMemcpyHostToDevice, c.stream),
       "copy");
    CK(cudaMemcpyAsync(c.d_pair_ent, pair_ent.data(), sizeof(int2) * c.nent, cudaMemcpyHostToDevice, c.stream),
       "copy");
    CK(cudaStreamSynchronize(c.stream), "create");
    c.stage = 1;
    return CCOV_OK;
}

ccov_status ccov_load(ccov_ctx* h, const double* cameras, const double* points, const ccov_obs* obs,
                      const double* obs_cov, int memory) {
    if (!h || !cameras || !points || !obs) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.stage < 1) return fail(&c, CCOV_ERR_INVALID_ARG, "context not created");
    if ((obs_cov != nullptr) != c.has_cov)
        return fail(&c, CCOV_ERR_INVALID_ARG, "obs_cov presence differs from ccov_create");
    if (memory == CCOV_MEM_HOST) {
        // the index set S must be the one the context was built for
        std::vector<int> pt_ptr, cam_ptr, cam_perm;
        std::vector<double> c9;
        const double* vc = cameras;
        if (c.opt.camera_model == CCOV_CAMERA_CENTRE8) {
            expand_centre(cameras, c.n, CCOV_MEM_HOST, c9);
            vc = c9.data();
        }
        ccov_status s = build_index(c, vc, points, obs, obs_cov, pt_ptr, cam_ptr, cam_perm);
        if (s != CCOV_OK) return s;
        std::vector<int> dptr(c.m + 1);
        CK(cudaMemcpy(dptr.data(), c.d_pt_ptr, sizeof(int) * (c.m + 1), cudaMemcpyDeviceToHost), "load");
        if (dptr != pt_ptr) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_load: index set differs");
    } else if (memory != CCOV_MEM_DEVICE) {
        return fail(&c, CCOV_ERR_INVALID_ARG, "unknown memory kind");
    }
    c.cov_ready = false;
    ccov_status s = upload(c, cameras, points, obs, obs_cov, memory);
    if (s != CCOV_OK) return s;
    c.stage = 1;
    c.null_done = false;
    return CCOV_OK;
}

}  // extern "C"

// ---------------------------------------------------------------------------
// Launch-only halves of the four steps: no host synchronisation, so that the
// batched form can run many contexts concurrently or capture them in a graph.
// Device-side errors land in the sticky flag and are read by check_device.
namespace {

void rec(Ctx& c, int i) {
    if (!c.capturing) cudaEventRecord(c.ev[i], c.stream);
}

ccov_status enq_information(Ctx& c) {
    c.launches = 0;
    CK(cudaMemsetAsync(c.d_flag, 0, 2 * sizeof(int), c.stream), "memset flag");
    ccov::launch_cam_prep(c);
    ccov::launch_point_info(c);
    ccov::launch_cam_info(c);
    CK(cudaGetLastError(), "ccov_information launch");
    return CCOV_OK;
}

ccov_status enq_schur(Ctx& c) {
    CK(cudaMemsetAsync(c.d_Z, 0, sizeof(double) * c.Np * c.Np, c.stream), "memset Z");
    CK(cudaMemsetAsync(c.d_W7, 0, sizeof(double) * 128, c.stream), "memset W7");
    ccov::launch_schur(c);
    CK(cudaGetLastError(), "ccov_schur launch");
    return CCOV_OK;
}

ccov_status enq_nullspace(Ctx& c, bool prep) {
    if (prep) ccov::launch_cam_prep(c);
    ccov::launch_nullspace(c, !prep);   // after step (a) on these inputs: its kept Jacobians
    CK(cudaGetLastError(), "ccov_nullspace launch");
    return CCOV_OK;
}

ccov_status factor_inverse_fp64(Ctx& c) {
    using ccov::kNB;
    const int64_t Np = c.Np, nb = Np / kNB;
    for (int64_t kb = 0; kb < nb; ++kb) {
        const int64_t k0 = kb * kNB, rem = Np - k0 - kNB;
        ccov::launch_potrf_diag(c, k0);
        if (rem > 0) {
            ccov::launch_copy_panel(c, k0);
            // L21 = A21 L_kk^-T
            ccov::prof_begin(c);
            ccov::launch_gemm64(c, true, false, rem, kNB, kNB, 1.0, c.d_P, kNB,
                                c.d_Linv + kb * kNB * kNB, kNB, 0.0, c.d_Z + (k0 + kNB) * Np + k0, Np, 0, 0);
            ccov::prof_end(c, 2.0 * rem * kNB * kNB);
            // A22 -= L21 L21^T (lower tiles)
            const double* L21 = c.d_Z + (k0 + kNB) * Np + k0;
            ccov::prof_begin(c);
            ccov::launch_gemm64(c, true, true, rem, rem, kNB, -1.0, L21, Np, L21, Np, 1.0,
                                c.d_Z + (k0 + kNB) * Np + k0 + kNB, Np, 0, 0);
            ccov::prof_end(c, (double)rem * (rem + 1) * kNB);
        }
    }
    rec(c, 3);
    CK(cudaMemsetAsync(c.d_R, 0, sizeof(double) * Np * Np, c.stream), "memset R");
    ccov::launch_init_identity(c, c.d_R, Np);
    for (int64_t kb = 0; kb < nb; ++kb) {
        const int64_t k0 = kb * kNB, rem = Np - k0 - kNB;
        ccov::launch_trtri_row(c, k0);
        if (rem > 0) {
            // R[k+1:, :k+1] -= L[k+1:, k] X[k, :k+1]
            ccov::prof_begin(c);
            ccov::launch_gemm64(c, false, false, rem, k0 + kNB, kNB, -1.0, c.d_Z + (k0 + kNB) * Np + k0, Np,
                                c.d_R + k0 * Np, Np, 1.0, c.d_R + (k0 + kNB) * Np, Np, 0, 0);
            ccov::prof_end(c, 2.0 * rem * (k0 + kNB) * kNB);
        }
    }
    return CCOV_OK;
}

ccov_status enq_covariance(Ctx& c, double* out, int out_memory) {
    ccov::launch_form_scaled(c);
    if (c.est_on && c.opt.precision == CCOV_PREC_FP64) ccov::est_keep_fp64(c);
    CK(cudaGetLastError(), "ccov_covariance launch");
    rec(c, 2);
    CK(cudaMemsetAsync(c.d_Sig, 0, sizeof(double) * 81 * c.n, c.stream), "memset");
    c.prof_used = 0;
    c.prof_flops = 0.0;
    if (c.opt.precision == CCOV_PREC_FP64) {
        ccov_status s = factor_inverse_fp64(c);
        if (s != CCOV_OK) return s;
    } else {
        cudaError_t e = ccov::mixed_factor_inverse(c);
        if (e != cudaSuccess) return cuda_fail(&c, e, "mixed path");
    }
    if (c.est_on) ccov::est_launch(c, ccov::mixed_inverse_factor(c));
    ccov::launch_extract(c);
    if (c.est_on) ccov::est_launch_final(c);
    CK(cudaGetLastError(), "ccov_covariance launch");
    if (out) {
        cudaMemcpyKind k = out_memory == CCOV_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CK(cudaMemcpyAsync(out, c.d_Sig, sizeof(double) * 81 * c.n, k, c.stream), "copy out");
    }
    return CCOV_OK;
}

void covariance_stats(Ctx& c) {
    c.stats.ms_covariance = elapsed(c, 0, 1);
    c.stats.ms_factor = elapsed(c, 2, 3);
    c.stats.ms_inverse = elapsed(c, 3, 1);
    c.stats.launches = c.launches;
    if (c.opt.profile) {
        double ms = 0.0;
        for (size_t k = 0; k + 1 < c.prof_used; k += 2) {
            float e = 0.f;
            cudaEventElapsedTime(&e, c.prof_ev[k], c.prof_ev[k + 1]);
            ms += e;
        }
        c.stats.ms_gemm = ms;
        c.stats.gemm_flops = c.prof_flops;
        c.stats.gemm_launches = (int64_t)(c.prof_used / 2);
    }
}

}  // namespace

extern "C" {

ccov_status ccov_information(ccov_ctx* h) {
    if (!h) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.stage < 1) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_information: context not created");
    c.cov_ready = false;
    rec(c, 0);
    ccov_status s = enq_information(c);
    if (s != CCOV_OK) return s;
    rec(c, 1);
    s = check_device(c, "ccov_information");
    if (s != CCOV_OK) return s;
    c.stats.ms_information = elapsed(c, 0, 1);
    c.stage = 2;
    return CCOV_OK;
}

ccov_status ccov_schur(ccov_ctx* h) {
    if (!h) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.stage < 2) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_schur: call ccov_information first");
    c.cov_ready = false;
    rec(c, 0);
    ccov_status s = enq_schur(c);
    if (s != CCOV_OK) return s;
    rec(c, 1);
    s = check_device(c, "ccov_schur");
    if (s != CCOV_OK) return s;
    c.stats.ms_schur = elapsed(c, 0, 1);
    c.stage = 3;
    return CCOV_OK;
}

ccov_status ccov_nullspace(ccov_ctx* h, double* H_P_out) {
    if (!h) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.stage < 1) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_nullspace: context not created");
    rec(c, 0);
    ccov_status s = enq_nullspace(c, c.stage < 2);
    if (s != CCOV_OK) return s;
    rec(c, 1);
    s = check_device(c, "ccov_nullspace");
    if (s != CCOV_OK) return s;
    c.stats.ms_nullspace = elapsed(c, 0, 1);
    if (H_P_out) CK(cudaMemcpy(H_P_out, c.d_HP, sizeof(double) * 63 * c.n, cudaMemcpyDeviceToHost), "copy H_P");
    c.null_done = true;
    return CCOV_OK;
}

ccov_status ccov_covariance(ccov_ctx* h, double* out, int out_memory, double* est_rel_err) {
    if (!h) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.stage < 3) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_covariance: call ccov_schur first");
    if (!c.null_done) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_covariance: call ccov_nullspace first");
    if (out_memory != CCOV_MEM_HOST && out_memory != CCOV_MEM_DEVICE)
        return fail(&c, CCOV_ERR_INVALID_ARG, "unknown memory kind");
    c.cov_ready = false;
    c.upd_norm_ok = false;
    c.est_on = est_rel_err != nullptr;
    c.est_k = (int)(c.opt.est_cameras < c.n ? c.opt.est_cameras : c.n);
    c.stats.est_cameras = 0;
    if (c.est_on) CK(ccov::est_alloc(c, c.est_k), "alloc error-estimate workspace");
    rec(c, 0);
    ccov_status s = enq_covariance(c, out, out_memory);
    c.stage = 2;  // Z is consumed in place
    if (s != CCOV_OK) { c.est_on = false; return s; }
    rec(c, 1);
    s = check_device(c, "ccov_covariance");
    if (s != CCOV_OK) { c.est_on = false; return s; }
    covariance_stats(c);
    c.cov_ready = true;
    if (c.est_on) {
        c.est_on = false;
        double est[3 * ccov::kEstMaxCams];
        CK(cudaMemcpy(est, c.d_est_out, sizeof(double) * 3 * c.est_k, cudaMemcpyDeviceToHost), "copy estimate");
        double worst = 0.0;
        for (int j = 0; j < c.est_k; ++j) worst = est[3 * j] > worst ? est[3 * j] : worst;
        for (int64_t i = 0; i < c.n; ++i) est_rel_err[i] = worst;
        c.stats.est_cameras = c.est_k;
        for (int j = 0; j < c.est_k; ++j) {
            const int64_t cam = (int64_t)est[3 * j + 2];
            est_rel_err[cam] = est[3 * j];
            c.stats.est_index[j] = cam;
            c.stats.est_rel[j] = est[3 * j];
            c.stats.est_norm[j] = est[3 * j + 1];
        }
    }
    return CCOV_OK;
}

ccov_status ccov_update_observations(ccov_ctx* h, const ccov_obs* add, int64_t k, const double* add_cov,
                                     double* out, int out_memory) {
    if (!h) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (!out || k < 0 || k > ccov::kUpdMaxObs || (k > 0 && !add))
        return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_update_observations: bad pointer or k");
    if (out_memory != CCOV_MEM_HOST && out_memory != CCOV_MEM_DEVICE)
        return fail(&c, CCOV_ERR_INVALID_ARG, "unknown memory kind");
    if (!c.cov_ready)
        return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_update_observations: call ccov_covariance first");
    if (c.opt.gauge != CCOV_GAUGE_NATURAL)
        return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_update_observations: natural gauge only");
    if ((add_cov != nullptr) != c.has_cov)
        return fail(&c, CCOV_ERR_INVALID_ARG, "add_cov presence differs from ccov_create");
    for (int64_t o = 0; o < k; ++o) {
        if (add[o].cam < 0 || add[o].cam >= c.n || add[o].pt < 0 || add[o].pt >= c.m)
            return fail(&c, CCOV_ERR_INVALID_ARG, "added observation %lld: index out of range", (long long)o);
        if (!std::isfinite(add[o].u[0]) || !std::isfinite(add[o].u[1]))
            return fail(&c, CCOV_ERR_INVALID_ARG, "added observation %lld: u not finite", (long long)o);
        if (add_cov) {
            const double* q = add_cov + 4 * o;
            if (!finite_all(q, 4) || !(q[0] > 0.0) || q[1] != q[2] || !(q[0] * q[3] - q[1] * q[2] > 0.0))
                return fail(&c, CCOV_ERR_INVALID_ARG, "added observation %lld: covariance not SPD", (long long)o);
        }
    }
    if (k == 0) {
        const cudaMemcpyKind kind = out_memory == CCOV_MEM_DEVICE ? cudaMemcpyDeviceToDevice : cudaMemcpyDeviceToHost;
        CK(cudaMemcpyAsync(out, c.d_Sig, sizeof(double) * 81 * c.n, kind, c.stream), "copy out");
        CK(cudaStreamSynchronize(c.stream), "ccov_update_observations");
        return CCOV_OK;
    }
    c.launches = 0;
    rec(c, 0);
    CK(ccov::update_enqueue(c, add, k, add_cov, out, out_memory), "ccov_update_observations");
    rec(c, 1);
    ccov_status s = check_device(c, "ccov_update_observations");
    if (s != CCOV_OK) return s;
    c.stats.ms_update = elapsed(c, 0, 1);
    c.stats.update_launches = c.launches;
    return CCOV_OK;
}

// ---------------------------------------------------------------------------
// Batched form: many independent scenes (sub-reconstructions, Sec. 5).
static ccov_status batch_check_args(ccov_ctx* const* ctxs, int k, double* const* outs) {
    if (!ctxs || !outs || k < 1) return CCOV_ERR_INVALID_ARG;
    for (int i = 0; i < k; ++i) {
        if (!ctxs[i] || !outs[i]) return CCOV_ERR_INVALID_ARG;
        if (ctxs[i]->c.stage < 1) return fail(&ctxs[i]->c, CCOV_ERR_INVALID_ARG, "batch: context not created");
    }
    return CCOV_OK;
}

static ccov_status batch_enqueue(Ctx& c, double* out, int out_memory) {
    c.est_on = false;
    c.cov_ready = false;
    rec(c, 0);
    ccov_status s = enq_information(c);
    if (s == CCOV_OK) s = enq_schur(c);
    if (s == CCOV_OK) s = enq_nullspace(c, false);
    if (s == CCOV_OK) s = enq_covariance(c, out, out_memory);
    rec(c, 1);
    return s;
}

ccov_status ccov_surrogate_features(ccov_ctx* h, float* features, double* scale) {
    if (!h || !features || !scale) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.stage < 2) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_surrogate_features: call ccov_information first");
    if (c.opt.camera_model != CCOV_CAMERA_RT9)
        return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_surrogate_features: the surrogate takes 9-value cameras");
    ccov::surr_launch_features(c, features, scale);
    CK(cudaGetLastError(), "ccov_surrogate_features launch");
    return check_device(c, "ccov_surrogate_features");
}

ccov_status ccov_surrogate_gauge_rows(ccov_ctx* h, const double* scale, double* q) {
    if (!h || !scale || !q) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.stage < 2) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_surrogate_gauge_rows: call ccov_information first");
    if (!c.null_done) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_surrogate_gauge_rows: call ccov_nullspace first");
    if (c.opt.camera_model != CCOV_CAMERA_RT9)
        return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_surrogate_gauge_rows: the surrogate takes 9-value cameras");
    ccov::surr_launch_gauge_rows(c, scale, q);
    CK(cudaGetLastError(), "ccov_surrogate_gauge_rows launch");
    return check_device(c, "ccov_surrogate_gauge_rows");
}

ccov_status ccov_batch_covariance(ccov_ctx* const* ctxs, int k, double* const* outs, int out_memory) {
    ccov_status s = batch_check_args(ctxs, k, outs);
    if (s != CCOV_OK) return s;
    if (out_memory != CCOV_MEM_HOST && out_memory != CCOV_MEM_DEVICE) return CCOV_ERR_INVALID_ARG;
    for (int i = 0; i < k; ++i) {
        s = batch_enqueue(ctxs[i]->c, outs[i], out_memory);
        if (s != CCOV_OK) return s;
    }
    ccov_status first = CCOV_OK;
    for (int i = 0; i < k; ++i) {
        Ctx& c = ctxs[i]->c;
        ccov_status si = check_device(c, "ccov_batch_covariance");
        c.stage = 2;
        c.null_done = true;
        if (si == CCOV_OK) covariance_stats(c);  // ms_covariance: the whole of steps (a)-(d)
        if (si != CCOV_OK && first == CCOV_OK) first = si;
    }
    return first;
}

}  // extern "C"

struct ccov_batch {
    std::vector<ccov_ctx*> ctxs;
    cudaStream_t master = nullptr;
    cudaEvent_t fork = nullptr;
    std::vector<cudaEvent_t> joins;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    ccov::GroupPlan* group = nullptr;   // the grouped form, or null (per scene)
    ccov_batch_info info{};
};

static void batch_free(ccov_batch* b) {
    if (!b) return;
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->group) ccov::group_free(b->group);
    for (auto e : b->joins)
        if (e) cudaEventDestroy(e);
    if (b->fork) cudaEventDestroy(b->fork);
    if (b->master) cudaStreamDestroy(b->master);
    delete b;
}

extern "C" {

// The grouped form: plan, autotune, one direct pass, then capture.
static ccov_status batch_create_grouped(ccov_ctx* const* ctxs, int k, double* const* outs_device, bool tune,
                                        ccov_batch** out) {
    std::vector<Ctx*> cs(k);
    for (int i = 0; i < k; ++i) cs[i] = &ctxs[i]->c;
    ccov_batch* b = new (std::nothrow) ccov_batch();
    if (!b) return CCOV_ERR_OOM;
    b->ctxs.assign(ctxs, ctxs + k);
    b->joins.assign(k, nullptr);
    bool ok = cudaStreamCreateWithFlags(&b->master, cudaStreamNonBlocking) == cudaSuccess;
    for (int i = 0; ok && i < k; ++i)
        ok = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { batch_free(b); return CCOV_ERR_CUDA; }
    cudaError_t e = ccov::group_create(cs.data(), outs_device, k, &b->group);
    if (e != cudaSuccess) { batch_free(b); return e == cudaErrorMemoryAllocation ? CCOV_ERR_OOM : CCOV_ERR_CUDA; }
    // inputs: after whatever the contexts' streams hold
    for (int i = 0; i < k; ++i) {
        cudaEventRecord(b->joins[i], cs[i]->stream);
        cudaStreamWaitEvent(b->master, b->joins[i], 0);
    }
    // one direct pass validates the scenes (and sets every kernel attribute)
    e = ccov::group_enqueue(*b->group, b->master);
    ccov_status s = e == cudaSuccess ? ccov::group_status(*b->group, b->master, "ccov_batch_create") : CCOV_ERR_CUDA;
    if (s != CCOV_OK) { batch_free(b); return s; }
    float tune_ms = 0.f;
    if (tune && ccov::group_autotune(*b->group, b->master, 1, &tune_ms) != cudaSuccess) {
        batch_free(b);
        return CCOV_ERR_CUDA;
    }
    s = ccov::group_status(*b->group, b->master, "ccov_batch_create");
    if (s != CCOV_OK) { batch_free(b); return s; }
    if (cudaStreamBeginCapture(b->master, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        batch_free(b);
        return CCOV_ERR_CUDA;
    }
    e = ccov::group_enqueue(*b->group, b->master);
    cudaError_t e2 = cudaStreamEndCapture(b->master, &b->graph);
    if (e != cudaSuccess || e2 != cudaSuccess) { batch_free(b); return CCOV_ERR_CUDA; }
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) { batch_free(b); return CCOV_ERR_CUDA; }
    b->info.form = CCOV_BATCH_GROUPED;
    b->info.launches = ccov::group_launches(*b->group);
    ccov::group_shape(*b->group, &b->info.gemm_ctas, &b->info.gemm_stages);
    b->info.tune_ms = tune_ms;
    *out = b;
    return CCOV_OK;
}

ccov_status ccov_batch_create(ccov_ctx* const* ctxs, int k, double* const* outs_device, ccov_batch** out) {
    return ccov_batch_create_ex(ctxs, k, outs_device, CCOV_BATCH_AUTO, out);
}

ccov_status ccov_batch_create_ex(ccov_ctx* const* ctxs, int k, double* const* outs_device, int form,
                                 ccov_batch** out) {
    if (!out) return CCOV_ERR_INVALID_ARG;
    *out = nullptr;
    const bool tune = !(form & CCOV_BATCH_NO_TUNE);
    form &= ~CCOV_BATCH_NO_TUNE;
    if (form != CCOV_BATCH_AUTO && form != CCOV_BATCH_PER_SCENE && form != CCOV_BATCH_GROUPED)
        return CCOV_ERR_INVALID_ARG;
    {
        ccov_status s0 = batch_check_args(ctxs, k, outs_device);
        if (s0 != CCOV_OK) return s0;
    }
    if (form != CCOV_BATCH_PER_SCENE) {
        std::vector<Ctx*> cs(k);
        for (int i = 0; i < k; ++i) cs[i] = &ctxs[i]->c;
        if (ccov::group_eligible(cs.data(), k)) return batch_create_grouped(ctxs, k, outs_device, tune, out);
        if (form == CCOV_BATCH_GROUPED)
            return fail(&ctxs[0]->c, CCOV_ERR_INVALID_ARG,
                        "grouped batch: every context needs MIXED precision with the same digits, nullspace "
                        "route and image-point model");
    }
    // one direct pass validates the scenes and sets every kernel attribute
    ccov_status s = ccov_batch_covariance(ctxs, k, outs_device, CCOV_MEM_DEVICE);
    if (s != CCOV_OK) return s;
    ccov_batch* b = new (std::nothrow) ccov_batch();
    if (!b) return CCOV_ERR_OOM;
    b->ctxs.assign(ctxs, ctxs + k);
    b->joins.assign(k, nullptr);
    bool ok = cudaStreamCreateWithFlags(&b->master, cudaStreamNonBlocking) == cudaSuccess &&
              cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming) == cudaSuccess;
    for (int i = 0; ok && i < k; ++i)
        ok = cudaEventCreateWithFlags(&b->joins[i], cudaEventDisableTiming) == cudaSuccess;
    if (!ok) { batch_free(b); return CCOV_ERR_CUDA; }
    // capture: fork every context's stream from the master stream, enqueue its
    // four steps, join back
    if (cudaStreamBeginCapture(b->master, cudaStreamCaptureModeThreadLocal) != cudaSuccess) {
        batch_free(b);
        return CCOV_ERR_CUDA;
    }
    cudaEventRecord(b->fork, b->master);
    for (int i = 0; i < k && s == CCOV_OK; ++i) {
        Ctx& c = ctxs[i]->c;
        cudaStreamWaitEvent(c.stream, b->fork, 0);
        c.capturing = true;
        s = batch_enqueue(c, outs_device[i], CCOV_MEM_DEVICE);
        c.capturing = false;
        cudaEventRecord(b->joins[i], c.stream);
        cudaStreamWaitEvent(b->master, b->joins[i], 0);
    }
    cudaError_t e = cudaStreamEndCapture(b->master, &b->graph);
    if (s != CCOV_OK || e != cudaSuccess) { batch_free(b); return s != CCOV_OK ? s : CCOV_ERR_CUDA; }
    if (cudaGraphInstantiate(&b->exec, b->graph, 0) != cudaSuccess) { batch_free(b); return CCOV_ERR_CUDA; }
    b->info.form = CCOV_BATCH_PER_SCENE;
    for (int i = 0; i < k; ++i) b->info.launches += ctxs[i]->c.launches;
    *out = b;
    return CCOV_OK;
}

ccov_status ccov_batch_get_info(const ccov_batch* b, ccov_batch_info* out) {
    if (!b || !out) return CCOV_ERR_INVALID_ARG;
    *out = b->info;
    return CCOV_OK;
}

ccov_status ccov_batch_run(ccov_batch* b, void* stream) {
    if (!b) return CCOV_ERR_INVALID_ARG;
    cudaStream_t st = stream ? static_cast<cudaStream_t>(stream) : b->master;
    // order the replay after whatever the contexts' streams hold (ccov_load copies)
    for (size_t i = 0; i < b->ctxs.size(); ++i) {
        if (cudaEventRecord(b->joins[i], b->ctxs[i]->c.stream) != cudaSuccess ||
            cudaStreamWaitEvent(st, b->joins[i], 0) != cudaSuccess)
            return CCOV_ERR_CUDA;
    }
    if (cudaGraphLaunch(b->exec, st) != cudaSuccess) return CCOV_ERR_CUDA;
    if (cudaStreamSynchronize(st) != cudaSuccess) return CCOV_ERR_CUDA;
    if (b->group) {
        ccov_status s = ccov::group_status(*b->group, st, "ccov_batch_run");
        if (s != CCOV_OK)
            for (ccov_ctx* h : b->ctxs) fail(&h->c, s, "ccov_batch_run: a scene of the grouped batch failed");
        return s;
    }
    ccov_status first = CCOV_OK;
    for (ccov_ctx* h : b->ctxs) {
        ccov_status si = check_device(h->c, "ccov_batch_run");
        if (si != CCOV_OK && first == CCOV_OK) first = si;
    }
    return first;
}

void ccov_batch_destroy(ccov_batch* b) { batch_free(b); }

ccov_status ccov_get_blocks(ccov_ctx* h, double* U, double* A_inv, double* W) {
    if (!h) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.stage < 2) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_get_blocks: call ccov_information first");
    if (U) {
        std::vector<double> u(45 * c.n);
        CK(cudaMemcpy(u.data(), c.d_U, 8 * u.size(), cudaMemcpyDeviceToHost), "copy U");
        for (int64_t i = 0; i < c.n; ++i) {
            int e = 0;
            for (int p = 0; p < 9; ++p)
                for (int q = 0; q <= p; ++q, ++e) {
                    U[81 * i + 9 * p + q] = u[45 * i + e];
                    U[81 * i + 9 * q + p] = u[45 * i + e];
                }
        }
    }
    if (A_inv) {
        std::vector<double> a(6 * c.m);
        CK(cudaMemcpy(a.data(), c.d_Ainv, 8 * a.size(), cudaMemcpyDeviceToHost), "copy A");
        for (int64_t j = 0; j < c.m; ++j) {
            const double* s = &a[6 * j];
            double full[9] = {s[0], s[1], s[2], s[1], s[3], s[4], s[2], s[4], s[5]};
            std::memcpy(A_inv + 9 * j, full, sizeof full);
        }
    }
    if (W) CK(cudaMemcpy(W, c.d_W, sizeof(double) * 27 * c.t, cudaMemcpyDeviceToHost), "copy W");
    return CCOV_OK;
}

ccov_status ccov_get_schur(ccov_ctx* h, double* Z, double* G, double* W7) {
    if (!h) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.stage < 3) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_get_schur: call ccov_schur first");
    if (Z)
        CK(cudaMemcpy2D(Z, sizeof(double) * c.N, c.d_Z, sizeof(double) * c.Np, sizeof(double) * c.N, c.N,
                        cudaMemcpyDeviceToHost), "copy Z");
    if (G) {
        std::vector<double> gp(7 * c.N), hp(63 * c.n);
        CK(cudaMemcpy(gp.data(), c.d_Gp, 8 * gp.size(), cudaMemcpyDeviceToHost), "copy G");
        if (c.null_done) CK(cudaMemcpy(hp.data(), c.d_HP, 8 * hp.size(), cudaMemcpyDeviceToHost), "copy H_P");
        for (size_t e = 0; e < gp.size(); ++e) G[e] = gp[e] + (c.null_done ? hp[e] : 0.0);
    }
    if (W7) {
        double w[49];
        CK(cudaMemcpy(w, c.d_W7, sizeof w, cudaMemcpyDeviceToHost), "copy W7");
        for (int p = 0; p < 7; ++p)
            for (int q = 0; q < 7; ++q) W7[7 * p + q] = p <= q ? w[7 * p + q] : w[7 * q + p];
    }
    return CCOV_OK;
}

ccov_status ccov_get_schur_blocks(ccov_ctx* h, const int64_t* ij, int64_t nblocks, double* out) {
    if (!h || nblocks < 0 || (nblocks > 0 && (!ij || !out))) return CCOV_ERR_INVALID_ARG;
    Ctx& c = h->c;
    if (c.stage < 3) return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_get_schur_blocks: call ccov_schur first");
    for (int64_t b = 0; b < nblocks; ++b) {
        const int64_t i = ij[2 * b], j = ij[2 * b + 1];
        if (i < 0 || j < 0 || i >= c.n || j > i)
            return fail(&c, CCOV_ERR_INVALID_ARG, "ccov_get_schur_blocks: need 0 <= j <= i < n");
        CK(cudaMemcpy2D(out + 81 * b, sizeof(double) * 9, c.d_Z + 9 * i * c.Np + 9 * j, sizeof(double) * c.Np,
                        sizeof(double) * 9, 9, cudaMemcpyDeviceToHost),
           "copy Z block");
    }
    return CCOV_OK;
}

ccov_status ccov_get_stats(const ccov_ctx* h, ccov_stats* out) {
    if (!h || !out) return CCOV_ERR_INVALID_ARG;
    *out = h->c.stats;
    return CCOV_OK;
}

void ccov_destroy(ccov_ctx* h) {
    if (!h) return;
    if (h->c.stream) cudaStreamSynchronize(h->c.stream);
    free_all(h->c);
    delete h;
}

}  // extern "C"
