// The batched form (Sec. 5, uncertainty for sub-reconstructions) as grouped
// launches: many scenes, every step of steps (a)-(d) one launch for all of
// them.
//
// Steps (a)-(c) run on the concatenation of the scenes (a "super-scene" with
// global camera, point and observation indices): their kernels work per
// point, observation or camera and need no change; the Schur blocks land in
// each scene's own dense matrix (per camera its scene, per scene the offset
// and leading dimension of its matrix) and the 7x7 sums are kept per scene.
// Step (d) (mixed precision) follows the single-scene schedule of
// mixed_factor_inverse sub-panel by sub-panel, in each scene's own groups of
// sub-panels; at each step every sub-step is one grouped launch over the
// scenes that have it (their
// parameter records and block prefixes were written to device memory when
// the plan was built), the trailing-update GEMMs as one persistent kernel
// over the tiles of all those scenes.  The Cholesky runs on one stream, the
// triangular inverse beside it on another, each step of the inverse after
// the same step of the Cholesky.  The whole sequence is recorded once as a
// CUDA graph of a few hundred nodes.
//
// A project-written autotuner picks the grouped GEMM's launch shape (the
// number of persistent CTAs and the pipeline depth) by timing the whole
// batch once per candidate when the plan is built.
#include <algorithm>
#include <cstring>
#include <vector>

#include "ccov_internal.cuh"
#include "group.cuh"

namespace ccov {
namespace {

constexpr int kFLq = 60, kFXq = 42;   // fixed points of Z_s / L and of X = L^-1 (k_mixed.cu)

struct GatherP {
    const double* cams;
    const double* pts;
    const ccov_obs* obs;
    const double* cov;
    int co, po;
};

// Inputs of every scene into the super-scene arrays (indices made global).
// Thread per item over the concatenated ranges: 9n camera values, 3m point
// values, t observations (and 4t covariance values).
__global__ void gather_kernel(int k, const GatherP* __restrict__ P, const int64_t* __restrict__ pc,
                              const int64_t* __restrict__ pp, const int64_t* __restrict__ po,
                              double* __restrict__ cams, double* __restrict__ pts, ccov_obs* __restrict__ obs,
                              double* __restrict__ cov) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    const int64_t nc = pc[k], np = pp[k], no = po[k];
    if (e < nc) {
        const int q = find_group(pc, k, e);
        cams[e] = P[q].cams[e - pc[q]];
    } else if (e < nc + np) {
        const int64_t f = e - nc;
        const int q = find_group(pp, k, f);
        pts[f] = P[q].pts[f - pp[q]];
    } else if (e < nc + np + no) {
        const int64_t f = e - nc - np;
        const int q = find_group(po, k, f);
        ccov_obs r = P[q].obs[f - po[q]];
        r.cam += P[q].co;
        r.pt += P[q].po;
        obs[f] = r;
        if (cov)
            for (int i = 0; i < 4; ++i) cov[4 * f + i] = P[q].cov[4 * (f - po[q]) + i];
    }
}

// out_q = the scene's rows of the global block array (81 values per camera).
__global__ void scatter_kernel(int k, const double* __restrict__ Sig, double* const* __restrict__ outs,
                               const int64_t* __restrict__ pre) {
    const int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x;
    if (e >= pre[k]) return;
    const int q = find_group(pre, k, e);
    outs[q][e - pre[q]] = Sig[e];
}

enum OpKind {
    OP_SLICE_ROWS, OP_SLICE_COLS, OP_POTRF, OP_GEMM, OP_GRAM, OP_ZSCALE, OP_IDENT, OP_RECORD, OP_WAIT
};

struct Op {
    int kind = 0, side = 0, K = 0, k = 0, ev = 0;
    size_t rec = 0, pre = 0;
    int64_t blocks = 0;
};

enum GBuf { G_P = 0, G_Q = 1, G_P2 = 2, G_Q2 = 3, G_L = 4 };

}  // namespace

struct GroupPlan {
    int k = 0, s = 5;
    std::vector<Ctx*> ctx;
    Ctx sup;   // the super-scene: its pointer fields address the concatenated arrays and arenas
    std::vector<int64_t> n, m, t, N, Np, nb, co, po, oo, zo, dofs, dig_off;
    long long* R = nullptr;
    __nv_bfloat16* dig[5] = {};
    int* ex[5] = {};
    CUtensorMap* h_maps = nullptr;   // per scene: Z, R, B of P, Q, P2, Q2, L
    std::vector<unsigned char> blob;
    unsigned char* d_blob = nullptr;
    std::vector<Op> ops;
    size_t gather_rec = 0, gather_pre = 0, scatter_pre = 0, scatter_outs = 0;
    size_t gauge_rec = 0, fd_rec = 0, fd_pre = 0, ex_rec = 0, ex_pre = 0;
    int64_t gather_blocks = 0, fd_blocks = 0, ex_blocks = 0, scatter_blocks = 0;
    cudaStream_t hi = nullptr, side = nullptr;
    std::vector<cudaEvent_t> ev;     // [0] fork, [1] Cholesky done, [2] inverse done, [3 + p] step p
    int gemm_cap = 0, gemm_stages = 0;
    int64_t launches = 0;
    std::vector<std::vector<size_t>> gemm_rec;   // per GEMM op: its problems (for re-tuning)

    template <class T>
    size_t put(const std::vector<T>& v) {
        size_t off = (blob.size() + 127) / 128 * 128;
        blob.resize(off + sizeof(T) * v.size());
        if (!v.empty()) std::memcpy(blob.data() + off, v.data(), sizeof(T) * v.size());
        return off;
    }
    template <class T>
    const T* at(size_t off) const { return reinterpret_cast<const T*>(d_blob + off); }

    long long* Zq(int q) const { return reinterpret_cast<long long*>(sup.d_Z + zo[q]); }
    long long* Rq(int q) const { return R + zo[q]; }
    __nv_bfloat16* D(int b, int q) const { return dig[b] + dig_off[q]; }
    int* E(int b, int q) const { return ex[b] + dofs[q]; }
};

namespace {

template <class T>
cudaError_t galloc(Ctx& c, T** p, size_t count) {
    cudaError_t e = cudaMalloc(reinterpret_cast<void**>(p), (count ? count : 1) * sizeof(T));
    if (e == cudaSuccess) c.bytes += (int64_t)(count * sizeof(T));
    return e;
}

// A grouped sub-step: the per-scene records and block counts of the scenes
// that have it.
template <class R>
struct Step {
    std::vector<R> rec;
    std::vector<int64_t> pre{0};
    void add(const R& r, int64_t blocks) {
        rec.push_back(r);
        pre.push_back(pre.back() + blocks);
    }
};

struct GemmStep {
    std::vector<GemmProblem> probs;
    int64_t pairs = 0;
};

}  // namespace

// ---------------------------------------------------------------------------
// Plan building: the same sequence as mixed_factor_inverse, per scene, merged
// by (window of sub-panel groups, sub-panel, sub-step).

namespace {

GemmProblem problem(const GroupPlan& P, int q, int K, int ba, int a_row0, int M, int bb, int b_row0, int N,
                    bool onR, int c_x0, int c_y0, int lower, int sub, int Fc, const int* expA, const int* expB) {
    GemmProblem g;
    std::memset(&g, 0, sizeof g);
    g.mapC = P.h_maps[7 * q + (onR ? 1 : 0)];
    g.mapB = P.h_maps[7 * q + 2 + bb];
    g.g.digA = P.D(ba, q);
    g.g.digB = P.D(bb, q);
    g.g.M = M;
    g.g.N = N;
    g.g.plane_rows = (int)P.Np[q];
    g.g.a_row0 = a_row0;
    g.g.b_row0 = b_row0;
    g.g.c_x0 = c_x0;
    g.g.c_y0 = c_y0;
    g.g.lower = lower;
    g.g.sub = sub;
    g.g.shift0 = Fc - 14;
    g.g.expA = expA;
    g.g.expB = expB;
    g.g.skip_fill = -1;
    (void)K;
    return g;
}

}  // namespace

static cudaError_t plan_ops(GroupPlan& P) {
    const int k = P.k, s = P.s;
    int64_t max_nb = 0;
    for (int q = 0; q < k; ++q) max_nb = std::max(max_nb, P.nb[q]);
    P.ev.assign(3 + (size_t)max_nb, nullptr);

    auto add_slice_rows = [&](int side, int K, Step<SliceRowsP>& st) {
        if (st.rec.empty()) return;
        Op o;
        o.kind = OP_SLICE_ROWS; o.side = side; o.K = K; o.k = (int)st.rec.size();
        o.rec = P.put(st.rec); o.pre = P.put(st.pre); o.blocks = st.pre.back();
        P.ops.push_back(o);
    };
    auto add_slice_cols = [&](int side, int K, Step<SliceColsP>& st) {
        if (st.rec.empty()) return;
        Op o;
        o.kind = OP_SLICE_COLS; o.side = side; o.K = K; o.k = (int)st.rec.size();
        o.rec = P.put(st.rec); o.pre = P.put(st.pre); o.blocks = st.pre.back();
        P.ops.push_back(o);
    };
    auto add_potrf = [&](std::vector<PotrfP>& v) {
        if (v.empty()) return;
        Op o;
        o.kind = OP_POTRF; o.k = (int)v.size(); o.rec = P.put(v);
        P.ops.push_back(o);
    };
    auto add_gram = [&](Step<GramP>& st) {
        if (st.rec.empty()) return;
        Op o;
        o.kind = OP_GRAM; o.side = 1; o.k = (int)st.rec.size();
        o.rec = P.put(st.rec); o.pre = P.put(st.pre); o.blocks = st.pre.back();
        P.ops.push_back(o);
    };
    auto add_gemm = [&](int side, int K, GemmStep& st) {
        if (st.probs.empty() || st.pairs == 0) return;
        Op o;
        o.kind = OP_GEMM; o.side = side; o.K = K; o.k = (int)st.probs.size();
        o.rec = P.put(st.probs); o.blocks = st.pairs;
        P.ops.push_back(o);
    };
    auto gemm_add = [&](GemmStep& st, const GemmProblem& pr) {
        const int64_t pairs = mixed_tile_pairs(pr.g.M, pr.g.N, pr.g.lower);
        if (pairs == 0) return;
        GemmProblem x = pr;
        x.pair0 = st.pairs;
        st.pairs += pairs;
        st.probs.push_back(x);
    };
    auto srows = [&](int q, int rows, const long long* src, int buf) {
        SliceRowsP r;
        r.src = src; r.ld = P.Np[q]; r.rows = rows; r.F = kFLq; r.s = s; r.plane_rows = (int)P.Np[q];
        r.dst = P.D(buf, q); r.expo = P.E(buf, q);
        return r;
    };
    auto scols = [&](int q, int ncols, const long long* src, int buf) {
        SliceColsP r;
        r.src = src; r.ld = P.Np[q]; r.ncols = ncols; r.F = kFXq; r.s = s; r.plane_rows = (int)P.Np[q];
        r.dst = P.D(buf, q); r.expo = P.E(buf, q);
        return r;
    };

    // ---- zscale, then the Cholesky on the high-priority stream ----
    {
        Step<ZscaleP> z;
        for (int q = 0; q < k; ++q) {
            ZscaleP r;
            r.N = P.N[q]; r.Np = P.Np[q]; r.nt = (P.Np[q] + 31) / 32;
            r.Z = P.sup.d_Z + P.zo[q]; r.F = P.sup.d_F + 7 * 9 * P.co[q]; r.G = P.sup.d_G + 7 * 9 * P.co[q];
            r.D = P.sup.d_D + P.dofs[q];
            z.add(r, r.nt * r.nt);
        }
        Op o;
        o.kind = OP_ZSCALE; o.k = k; o.rec = P.put(z.rec); o.pre = P.put(z.pre); o.blocks = z.pre.back();
        P.ops.push_back(o);
    }
    const int kN = kNB;
    // Sub-panel groups as in mixed_factor_inverse: per scene, m = its
    // mixed_group_max (4 or 2) while that many are left, else 2, else 1.
    // Group starts lie in windows of gmax sub-panels (the largest group of
    // any scene); slot j of a window holds, for every scene with sub-panel
    // j, exactly the single-scene operations of j, so each scene's
    // arithmetic (and result) is the single-scene one.
    int64_t gmax = 2;
    for (int q = 0; q < k; ++q) gmax = std::max(gmax, mixed_group_max(s, P.nb[q]));
    auto group_of = [&](int64_t nbq, int64_t j, int64_t& gs, int64_t& m) {
        const int64_t gq = mixed_group_max(s, nbq);
        gs = 0;
        for (;;) {
            const int64_t left = nbq - gs;
            m = left >= gq ? gq : (left >= 2 ? 2 : 1);
            if (j < gs + m) return;
            gs += m;
        }
    };
    const int kKs[3] = {128, 256, 512};
    auto kidx = [&](int64_t K) { return K == 128 ? 0 : (K == 256 ? 1 : 2); };
    for (int64_t p = 0; p < max_nb; p += gmax) {
        for (int64_t j = p; j < p + gmax; ++j) {
            const int64_t kj = j * kN;
            std::vector<PotrfP> pot;
            Step<SliceRowsP> s1, s2, s4[3];
            GemmStep g1, g2, g4[3];
            for (int q = 0; q < k; ++q) {
                if (P.nb[q] <= j) continue;
                const int64_t Npq = P.Np[q], remJ = Npq - kj - kN;
                int64_t gs, m;
                group_of(P.nb[q], j, gs, m);
                pot.push_back({P.Zq(q), Npq, kj, P.D(G_L, q), P.E(G_L, q), s});
                if (remJ <= 0) continue;
                const long long* colj = P.Zq(q) + (kj + kN) * Npq + kj;
                // L[rows > j, j] = A[rows > j, j] L_jj^-T
                s1.add(srows(q, (int)remJ, colj, G_P), grp_slice_rows_blocks(128, (int)remJ));
                gemm_add(g1, problem(P, q, 128, G_P, 0, (int)remJ, G_L, (int)kj, kN, false, (int)kj, (int)(kj + kN), 0,
                                     0, kFLq, nullptr, P.E(G_L, q)));
                // the group's later columns
                const int64_t w = gs + m - 1 - j;
                if (w > 0) {
                    s2.add(srows(q, (int)remJ, colj, G_P), grp_slice_rows_blocks(128, (int)remJ));
                    gemm_add(g2, problem(P, q, 128, G_P, 0, (int)remJ, G_P, 0, (int)(w * kN), false, (int)(kj + kN),
                                         (int)(kj + kN), 1, 1, kFLq, nullptr, nullptr));
                }
                // after the group's last sub-panel: its trailing update (K = 128 m)
                const int64_t kg = (gs + m) * kN, remG = Npq - kg;
                if (j == gs + m - 1 && remG > 0) {
                    const int K = (int)(m * kN), x = kidx(K);
                    s4[x].add(srows(q, (int)remG, P.Zq(q) + kg * Npq + gs * kN, G_P),
                              grp_slice_rows_blocks(K, (int)remG));
                    gemm_add(g4[x], problem(P, q, K, G_P, 0, (int)remG, G_P, 0, (int)remG, false, (int)kg, (int)kg, 1,
                                            1, kFLq, nullptr, nullptr));
                }
            }
            add_potrf(pot);
            add_slice_rows(0, 128, s1);
            add_gemm(0, 128, g1);
            add_slice_rows(0, 128, s2);
            add_gemm(0, 128, g2);
            for (int x = 0; x < 3; ++x) add_slice_rows(0, kKs[x], s4[x]);
            if (j == p + gmax - 1) {
                // the window's columns of L are final once its last trailing
                // updates are issued: they only write columns beyond it
                Op rec;
                rec.kind = OP_RECORD; rec.ev = 3 + (int)(p / gmax);
                P.ops.push_back(rec);
            }
            for (int x = 0; x < 3; ++x) add_gemm(0, kKs[x], g4[x]);
        }
    }
    {
        Op rec;
        rec.kind = OP_RECORD; rec.ev = 1;
        P.ops.push_back(rec);
    }
    // ---- the triangular inverse on the low-priority stream ----
    {
        Step<IdentP> id;
        for (int q = 0; q < k; ++q) id.add({P.Np[q], P.Rq(q)}, (P.Np[q] + 255) / 256);
        Op o;
        o.kind = OP_IDENT; o.side = 1; o.k = k; o.rec = P.put(id.rec); o.pre = P.put(id.pre); o.blocks = id.pre.back();
        P.ops.push_back(o);
    }
    for (int64_t p = 0; p < max_nb; p += gmax) {
        Op wt;
        wt.kind = OP_WAIT; wt.side = 1; wt.ev = 3 + (int)(p / gmax);
        P.ops.push_back(wt);
        for (int64_t j = p; j < p + gmax; ++j) {
            const int64_t kj = j * kN, ncj = kj + kN;
            Step<SliceColsP> c1, c2, c5[3];
            Step<SliceRowsP> r2, r5[3];
            Step<GramP> gr1;
            GemmStep f1, m2, m5[3];
            for (int q = 0; q < k; ++q) {
                if (P.nb[q] <= j) continue;
                const int64_t Npq = P.Np[q];
                int64_t gs, m;
                group_of(P.nb[q], j, gs, m);
                // finalize(j): X[j, :ncj] = L_jj^-1 R[j, :ncj], Gram blocks
                c1.add(scols(q, (int)ncj, P.Rq(q) + kj * Npq, G_Q2), grp_slice_cols_blocks((int)ncj));
                gemm_add(f1, problem(P, q, 128, G_L, (int)kj, kN, G_Q2, 0, (int)ncj, true, 0, (int)kj, 0, 0, kFXq,
                                     P.E(G_L, q), P.E(G_Q2, q)));
                gr1.add({P.n[q], Npq, kj, ncj, P.Rq(q), P.sup.d_Sig + 81 * P.co[q]}, grp_gram_blocks(ncj));
                // the group's later rows: R[j+1 .. gs+m-1, :ncj] -= L[j+1 .. gs+m-1, j] X[j, :ncj]
                const int64_t w = gs + m - 1 - j;
                if (w > 0) {
                    c2.add(scols(q, (int)ncj, P.Rq(q) + kj * Npq, G_Q2), grp_slice_cols_blocks((int)ncj));
                    r2.add(srows(q, (int)(w * kN), P.Zq(q) + (kj + kN) * Npq + kj, G_P2),
                           grp_slice_rows_blocks(128, (int)(w * kN)));
                    gemm_add(m2, problem(P, q, 128, G_P2, 0, (int)(w * kN), G_Q2, 0, (int)ncj, true, 0, (int)(kj + kN),
                                         0, 1, kFXq, nullptr, P.E(G_Q2, q)));
                }
                // after the group: R[rows >= kg, :kg] -= L[rows >= kg, group] X[group, :kg]  (K = 128 m)
                const int64_t kg = (gs + m) * kN, remG = Npq - kg;
                if (j == gs + m - 1 && remG > 0) {
                    const int K = (int)(m * kN), x = kidx(K);
                    c5[x].add(scols(q, (int)kg, P.Rq(q) + gs * kN * Npq, G_Q2), grp_slice_cols_blocks((int)kg));
                    r5[x].add(srows(q, (int)remG, P.Zq(q) + kg * Npq + gs * kN, G_P2),
                              grp_slice_rows_blocks(K, (int)remG));
                    gemm_add(m5[x], problem(P, q, K, G_P2, 0, (int)remG, G_Q2, 0, (int)kg, true, 0, (int)kg, 0, 1,
                                            kFXq, nullptr, P.E(G_Q2, q)));
                }
            }
            add_slice_cols(1, 128, c1);
            add_gemm(1, 128, f1);
            add_gram(gr1);
            add_slice_cols(1, 128, c2);
            add_slice_rows(1, 128, r2);
            add_gemm(1, 128, m2);
            for (int x = 0; x < 3; ++x) {
                add_slice_cols(1, kKs[x], c5[x]);
                add_slice_rows(1, kKs[x], r5[x]);
                add_gemm(1, kKs[x], m5[x]);
            }
        }
    }
    Op rec;
    rec.kind = OP_RECORD; rec.side = 1; rec.ev = 2;
    P.ops.push_back(rec);
    return cudaSuccess;
}

// ---------------------------------------------------------------------------
static void run_ops(GroupPlan& P) {
    int* flag = P.sup.d_flag;
    for (const Op& o : P.ops) {
        cudaStream_t st = o.side ? P.side : P.hi;
        switch (o.kind) {
            case OP_SLICE_ROWS:
                grp_slice_rows(st, o.K, P.at<SliceRowsP>(o.rec), P.at<int64_t>(o.pre), o.k, o.blocks, flag);
                break;
            case OP_SLICE_COLS:
                grp_slice_cols(st, o.K, P.at<SliceColsP>(o.rec), P.at<int64_t>(o.pre), o.k, o.blocks, flag);
                break;
            case OP_POTRF: grp_potrf(st, P.at<PotrfP>(o.rec), o.k, flag); break;
            case OP_GEMM:
                grp_gemm(st, P.s, o.K, P.at<GemmProblem>(o.rec), o.k, o.blocks, flag, P.gemm_cap, P.gemm_stages);
                break;
            case OP_GRAM: grp_gram(st, P.at<GramP>(o.rec), P.at<int64_t>(o.pre), o.k, o.blocks); break;
            case OP_ZSCALE: grp_zscale(st, P.at<ZscaleP>(o.rec), P.at<int64_t>(o.pre), o.k, o.blocks, flag); break;
            case OP_IDENT: grp_identity(st, P.at<IdentP>(o.rec), P.at<int64_t>(o.pre), o.k, o.blocks); break;
            case OP_RECORD: cudaEventRecord(P.ev[o.ev], st); continue;
            case OP_WAIT: cudaStreamWaitEvent(st, P.ev[o.ev], 0); continue;
        }
        P.launches++;
    }
}

// Steps (a)-(d) of every scene, enqueued on `main` (and forked onto the two
// streams of step (d)); no host synchronisation, so it can be captured.
cudaError_t group_enqueue(GroupPlan& P, cudaStream_t main) {
    Ctx& c = P.sup;
    c.stream = main;
    P.launches = 0;
    cudaError_t e;
    if ((e = cudaMemsetAsync(c.d_flag, 0, 2 * sizeof(int), main)) != cudaSuccess) return e;
    gather_kernel<<<(unsigned)P.gather_blocks, 256, 0, main>>>(P.k, P.at<GatherP>(P.gather_rec),
                                                                P.at<int64_t>(P.gather_pre),
                                                                P.at<int64_t>(P.gather_pre) + (P.k + 1),
                                                                P.at<int64_t>(P.gather_pre) + 2 * (P.k + 1), c.d_cams,
                                                                c.d_pts, c.d_obs, c.d_obscov);
    P.launches++;
    // steps (a)-(c) on the super-scene
    c.launches = 0;
    launch_cam_prep(c);
    launch_point_info(c);
    launch_cam_info(c);
    int64_t zsum = 0;
    for (int q = 0; q < P.k; ++q) zsum += P.Np[q] * P.Np[q];
    if ((e = cudaMemsetAsync(c.d_Z, 0, sizeof(double) * zsum, main)) != cudaSuccess) return e;
    if ((e = cudaMemsetAsync(c.d_W7, 0, sizeof(double) * 128 * P.k, main)) != cudaSuccess) return e;
    launch_schur(c);
    launch_nullspace(c, true);
    launch_g(c);
    grp_gauge(main, P.at<GaugeP>(P.gauge_rec), P.k, c.d_flag);
    grp_fd(main, P.at<FdP>(P.fd_rec), P.at<int64_t>(P.fd_pre), P.k, P.fd_blocks, c.d_flag);
    if ((e = cudaMemsetAsync(c.d_Sig, 0, sizeof(double) * 81 * c.n, main)) != cudaSuccess) return e;
    P.launches += c.launches + 2;
    // step (d): fork onto the Cholesky and inverse streams
    if ((e = cudaEventRecord(P.ev[0], main)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(P.hi, P.ev[0], 0)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(P.side, P.ev[0], 0)) != cudaSuccess) return e;
    int64_t rsum = zsum;
    if ((e = cudaMemsetAsync(P.R, 0, sizeof(long long) * rsum, P.side)) != cudaSuccess) return e;
    run_ops(P);
    if ((e = cudaStreamWaitEvent(main, P.ev[1], 0)) != cudaSuccess) return e;
    if ((e = cudaStreamWaitEvent(main, P.ev[2], 0)) != cudaSuccess) return e;
    grp_extract(main, P.at<ExtractP>(P.ex_rec), P.at<int64_t>(P.ex_pre), P.k, P.ex_blocks);
    scatter_kernel<<<(unsigned)P.scatter_blocks, 256, 0, main>>>(
        P.k, c.d_Sig, reinterpret_cast<double* const*>(P.d_blob + P.scatter_outs), P.at<int64_t>(P.scatter_pre));
    P.launches += 2;
    return cudaGetLastError();
}

void group_free(GroupPlan* P) {
    if (!P) return;
    Ctx& c = P->sup;
    if (P->hi) cudaStreamSynchronize(P->hi);
    if (P->side) cudaStreamSynchronize(P->side);
    void* ptrs[] = {c.d_cams, c.d_pts, c.d_obs, c.d_obscov, c.d_pt_ptr, c.d_cam_ptr, c.d_cam_perm, c.d_camprep,
                    c.d_W, c.d_Ainv, c.d_U, c.d_V, c.d_J, c.d_pair_desc, c.d_pair_ent, c.d_w7part, c.d_Z, c.d_Gp, c.d_W7,
                    c.d_HP, c.d_F, c.d_G, c.d_D, c.d_Sig, c.d_small, c.d_flag, P->R, P->d_blob,
                    const_cast<int*>(c.d_cam_scene), const_cast<int64_t*>(c.d_scene_zo),
                    const_cast<int64_t*>(c.d_scene_ld), const_cast<int*>(c.d_scene_co),
                    const_cast<int*>(c.d_scene_po), const_cast<int64_t*>(c.d_scene_wpo)};
    for (void* p : ptrs)
        if (p) cudaFree(p);
    for (int b = 0; b < 5; ++b) {
        if (P->dig[b]) cudaFree(P->dig[b]);
        if (P->ex[b]) cudaFree(P->ex[b]);
    }
    for (auto e : P->ev)
        if (e) cudaEventDestroy(e);
    if (P->hi) cudaStreamDestroy(P->hi);
    if (P->side) cudaStreamDestroy(P->side);
    delete[] P->h_maps;
    c.d_cam_scene = nullptr;
    delete P;
}

// Scenes that can share one plan: mixed precision with the same digits,
// nullspace route, image-point model (sigma or per-observation covariance).
bool group_eligible(Ctx* const* ctxs, int k) {
    if (k < 1) return false;
    const Ctx& a = *ctxs[0];
    for (int q = 0; q < k; ++q) {
        const Ctx& b = *ctxs[q];
        if (b.opt.precision != CCOV_PREC_MIXED || b.opt.mixed_slices != a.opt.mixed_slices ||
            b.opt.nullspace_route != a.opt.nullspace_route || b.has_cov != a.has_cov ||
            b.opt.gauge != CCOV_GAUGE_NATURAL || b.opt.camera_model != a.opt.camera_model ||
            (!a.has_cov && b.sigma != a.sigma))
            return false;
    }
    return true;
}

cudaError_t group_create(Ctx* const* ctxs, double* const* outs, int k, GroupPlan** out) {
    *out = nullptr;
    GroupPlan* Pp = new GroupPlan();
    GroupPlan& P = *Pp;
    P.k = k;
    P.s = ctxs[0]->opt.mixed_slices;
    P.ctx.assign(ctxs, ctxs + k);
    Ctx& c = P.sup;
    c.opt = ctxs[0]->opt;
    c.sigma = ctxs[0]->sigma;
    c.has_cov = ctxs[0]->has_cov;
    cudaError_t e = cudaSuccess;
#define GCK(x)                        \
    do {                              \
        if ((e = (x)) != cudaSuccess) { \
            group_free(Pp);           \
            return e;                 \
        }                             \
    } while (0)
    // sizes and offsets
    int64_t ns = 0, ms = 0, ts = 0, zs = 0, ds = 0, dg = 0, np = 0, ne = 0;
    for (int q = 0; q < k; ++q) {
        const Ctx& x = *ctxs[q];
        P.n.push_back(x.n); P.m.push_back(x.m); P.t.push_back(x.t); P.N.push_back(x.N); P.Np.push_back(x.Np);
        P.nb.push_back(x.Np / kNB);
        P.co.push_back(ns); P.po.push_back(ms); P.oo.push_back(ts); P.zo.push_back(zs); P.dofs.push_back(ds);
        P.dig_off.push_back(dg);
        ns += x.n; ms += x.m; ts += x.t; zs += x.Np * x.Np; ds += x.Np; dg += (int64_t)P.s * x.Np * kGroupDigitK;
        np += x.npairs; ne += x.nent;
    }
    P.co.push_back(ns); P.po.push_back(ms); P.oo.push_back(ts);
    c.n = ns; c.m = ms; c.t = ts; c.N = 9 * ns; c.Np = 0; c.npairs = np; c.nent = ne; c.nscenes = k;
    // per scene the same W7 partial sums as on its own (warps by its point
    // count), so that every scene's sums run in the same order
    std::vector<int64_t> wpo(k + 1, 0);
    for (int q = 0; q < k; ++q) wpo[q + 1] = wpo[q] + w7_warps_for(ctxs[q]->m);
    c.w7_total = wpo[k];
    // index arrays of the super-scene, from each context's device copies
    std::vector<int> pt_ptr(ms + 1, 0), cam_ptr(ns + 1, 0), cam_perm(ts), cam_scene(ns), sco(k), spo(k + 1);
    std::vector<int4> desc;
    std::vector<int2> ent;
    std::vector<int64_t> szo(k), sld(k);
    for (int q = 0; q < k; ++q) {
        const Ctx& x = *ctxs[q];
        std::vector<int> a(x.m + 1), b(x.n + 1), pm(x.t);
        std::vector<int4> d(x.npairs);
        std::vector<int2> en(x.nent);
        GCK(cudaMemcpy(a.data(), x.d_pt_ptr, sizeof(int) * a.size(), cudaMemcpyDeviceToHost));
        GCK(cudaMemcpy(b.data(), x.d_cam_ptr, sizeof(int) * b.size(), cudaMemcpyDeviceToHost));
        GCK(cudaMemcpy(pm.data(), x.d_cam_perm, sizeof(int) * pm.size(), cudaMemcpyDeviceToHost));
        GCK(cudaMemcpy(d.data(), x.d_pair_desc, sizeof(int4) * d.size(), cudaMemcpyDeviceToHost));
        GCK(cudaMemcpy(en.data(), x.d_pair_ent, sizeof(int2) * en.size(), cudaMemcpyDeviceToHost));
        for (int64_t j = 1; j <= x.m; ++j) pt_ptr[P.po[q] + j] = a[j] + (int)P.oo[q];
        for (int64_t i = 1; i <= x.n; ++i) cam_ptr[P.co[q] + i] = b[i] + (int)P.oo[q];
        for (int64_t o = 0; o < x.t; ++o) cam_perm[P.oo[q] + o] = pm[o] + (int)P.oo[q];
        for (int64_t i = 0; i < x.n; ++i) cam_scene[P.co[q] + i] = q;
        const int base = (int)ent.size();
        for (const int4& v : d) desc.push_back(make_int4(v.x + (int)P.co[q], v.y + (int)P.co[q], v.z + base, v.w));
        for (const int2& v : en) ent.push_back(make_int2(v.x + (int)P.oo[q], v.y + (int)P.oo[q]));
        sco[q] = (int)P.co[q];
        spo[q] = (int)P.po[q];
        szo[q] = P.zo[q];
        sld[q] = P.Np[q];
    }
    spo[k] = (int)ms;
    // super-scene arrays and arenas
    GCK(galloc(c, &c.d_cams, 9 * ns)); GCK(galloc(c, &c.d_pts, 3 * ms)); GCK(galloc(c, &c.d_obs, ts));
    if (c.has_cov) GCK(galloc(c, &c.d_obscov, 4 * ts));
    GCK(galloc(c, &c.d_pt_ptr, ms + 1)); GCK(galloc(c, &c.d_cam_ptr, ns + 1)); GCK(galloc(c, &c.d_cam_perm, ts));
    GCK(galloc(c, &c.d_camprep, kCamPrep * ns)); GCK(galloc(c, &c.d_W, 27 * ts)); GCK(galloc(c, &c.d_Ainv, 6 * ms));
    GCK(galloc(c, &c.d_U, 45 * ns)); GCK(galloc(c, &c.d_V, 27 * ts)); GCK(galloc(c, &c.d_J, 24 * ts));
    GCK(galloc(c, &c.d_pair_desc, np)); GCK(galloc(c, &c.d_pair_ent, ne));
    GCK(galloc(c, &c.d_w7part, (size_t)56 * c.w7_total));
    GCK(galloc(c, &c.d_Z, zs)); GCK(galloc(c, &c.d_Gp, 7 * 9 * ns)); GCK(galloc(c, &c.d_W7, 128 * k));
    GCK(galloc(c, &c.d_HP, 63 * ns)); GCK(galloc(c, &c.d_F, 7 * 9 * ns)); GCK(galloc(c, &c.d_G, 7 * 9 * ns));
    GCK(galloc(c, &c.d_D, ds)); GCK(galloc(c, &c.d_Sig, 81 * ns)); GCK(galloc(c, &c.d_small, 128 * k));
    GCK(galloc(c, &c.d_flag, 2));
    GCK(galloc(c, &P.R, zs));
    for (int b = 0; b < 5; ++b) {
        GCK(galloc(c, &P.dig[b], dg));
        GCK(galloc(c, &P.ex[b], ds));
        GCK(cudaMemset(P.dig[b], 0, sizeof(__nv_bfloat16) * dg));
    }
    int *d_cs, *d_sco, *d_spo;
    int64_t *d_szo, *d_sld;
    GCK(galloc(c, &d_cs, ns)); c.d_cam_scene = d_cs;
    GCK(galloc(c, &d_szo, k)); c.d_scene_zo = d_szo;
    GCK(galloc(c, &d_sld, k)); c.d_scene_ld = d_sld;
    GCK(galloc(c, &d_sco, k)); c.d_scene_co = d_sco;
    GCK(galloc(c, &d_spo, k + 1)); c.d_scene_po = d_spo;
    {
        int64_t* d_wpo = nullptr;
        GCK(galloc(c, &d_wpo, k + 1));
        c.d_scene_wpo = d_wpo;
        GCK(cudaMemcpy(d_wpo, wpo.data(), sizeof(int64_t) * (k + 1), cudaMemcpyHostToDevice));
    }
    GCK(cudaMemcpy(c.d_pt_ptr, pt_ptr.data(), sizeof(int) * pt_ptr.size(), cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(c.d_cam_ptr, cam_ptr.data(), sizeof(int) * cam_ptr.size(), cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(c.d_cam_perm, cam_perm.data(), sizeof(int) * cam_perm.size(), cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(c.d_pair_desc, desc.data(), sizeof(int4) * desc.size(), cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(c.d_pair_ent, ent.data(), sizeof(int2) * ent.size(), cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(d_cs, cam_scene.data(), sizeof(int) * ns, cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(d_szo, szo.data(), sizeof(int64_t) * k, cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(d_sld, sld.data(), sizeof(int64_t) * k, cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(d_sco, sco.data(), sizeof(int) * k, cudaMemcpyHostToDevice));
    GCK(cudaMemcpy(d_spo, spo.data(), sizeof(int) * (k + 1), cudaMemcpyHostToDevice));
    // tensor maps per scene
    P.h_maps = new CUtensorMap[7 * (size_t)k];
    for (int q = 0; q < k; ++q) {
        bool ok = mixed_make_c_map(&P.h_maps[7 * q], P.Zq(q), P.Np[q], P.Np[q], P.Np[q]) &&
                  mixed_make_c_map(&P.h_maps[7 * q + 1], P.Rq(q), P.Np[q], P.Np[q], P.Np[q]);
        for (int b = 0; b < 5 && ok; ++b) ok = mixed_make_b_map(&P.h_maps[7 * q + 2 + b], P.D(b, q), P.s, P.Np[q]);
        if (!ok) { group_free(Pp); return cudaErrorInvalidValue; }
    }
    // records of the fixed launches
    {
        std::vector<GatherP> g(k);
        std::vector<int64_t> pc(k + 1, 0), pp(k + 1, 0), po(k + 1, 0);
        for (int q = 0; q < k; ++q) {
            const Ctx& x = *ctxs[q];
            g[q] = {x.d_cams, x.d_pts, x.d_obs, x.d_obscov, (int)P.co[q], (int)P.po[q]};
            pc[q + 1] = pc[q] + 9 * x.n;
            pp[q + 1] = pp[q] + 3 * x.m;
            po[q + 1] = po[q] + x.t;
        }
        std::vector<int64_t> all(pc);
        all.insert(all.end(), pp.begin(), pp.end());
        all.insert(all.end(), po.begin(), po.end());
        P.gather_rec = P.put(g);
        P.gather_pre = P.put(all);
        P.gather_blocks = (pc[k] + pp[k] + po[k] + 255) / 256;
        std::vector<GaugeP> ga(k);
        Step<FdP> fd;
        Step<ExtractP> ex;
        std::vector<int64_t> sp(k + 1, 0);
        std::vector<double*> o(outs, outs + k);
        for (int q = 0; q < k; ++q) {
            const int64_t r0 = 9 * P.co[q];
            double* Zs = c.d_Z + P.zo[q];
            ga[q] = {P.N[q], P.Np[q], c.d_G + 7 * r0, c.d_HP + 7 * r0, Zs, c.d_W7 + 128 * q, c.d_small + 128 * q};
            fd.add({P.N[q], P.Np[q], c.d_small + 128 * q, Zs, c.d_G + 7 * r0, c.d_F + 7 * r0, c.d_D + P.dofs[q]},
                   (P.Np[q] + 255) / 256);
            ex.add({P.n[q], c.d_D + P.dofs[q], c.d_HP + 63 * P.co[q], c.d_small + 128 * q + 49,
                    c.d_Sig + 81 * P.co[q]},
                   (P.n[q] * 81 + 255) / 256);
            sp[q + 1] = sp[q] + 81 * P.n[q];
        }
        P.gauge_rec = P.put(ga);
        P.fd_rec = P.put(fd.rec); P.fd_pre = P.put(fd.pre); P.fd_blocks = fd.pre.back();
        P.ex_rec = P.put(ex.rec); P.ex_pre = P.put(ex.pre); P.ex_blocks = ex.pre.back();
        P.scatter_pre = P.put(sp); P.scatter_outs = P.put(o); P.scatter_blocks = (sp[k] + 255) / 256;
    }
    GCK(plan_ops(P));
    GCK(galloc(c, &P.d_blob, P.blob.size()));
    GCK(cudaMemcpy(P.d_blob, P.blob.data(), P.blob.size(), cudaMemcpyHostToDevice));
    int lo = 0, hi = 0;
    GCK(cudaDeviceGetStreamPriorityRange(&lo, &hi));
    GCK(cudaStreamCreateWithPriority(&P.hi, cudaStreamNonBlocking, hi));
    GCK(cudaStreamCreateWithPriority(&P.side, cudaStreamNonBlocking, lo));
    for (auto& ev : P.ev) GCK(cudaEventCreateWithFlags(&ev, cudaEventDisableTiming));
    GCK(mixed_setup());
    GCK(setup_dense64());
    P.gemm_cap = 1 << 20;
    P.gemm_stages = mixed_stages(P.s);
#undef GCK
    *out = Pp;
    return cudaSuccess;
}

// The autotuner: every candidate launch shape of the grouped GEMMs (CTA
// count x pipeline depth) runs the whole batch `reps` times on `st`; the
// fastest is kept.  Returns the chosen shape's time per batch (ms).
cudaError_t group_autotune(GroupPlan& P, cudaStream_t st, int reps, float* best_ms) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    const int base = mixed_stages(P.s);
    const int caps[3] = {sms, sms * 3 / 4 / 2 * 2, sms / 2 / 2 * 2};
    const int stg[2] = {base, base - 1};
    cudaEvent_t a, b;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    float best = 1e30f;
    int bc = sms, bs = base;
    cudaError_t e = cudaSuccess;
    for (int ci = 0; ci < 3 && e == cudaSuccess; ++ci)
        for (int si = 0; si < 2 && e == cudaSuccess; ++si) {
            P.gemm_cap = caps[ci];
            P.gemm_stages = stg[si];
            cudaEventRecord(a, st);
            for (int r = 0; r < reps && e == cudaSuccess; ++r) e = group_enqueue(P, st);
            cudaEventRecord(b, st);
            if (e == cudaSuccess) e = cudaEventSynchronize(b);
            float ms = 0.f;
            cudaEventElapsedTime(&ms, a, b);
            ms /= (float)reps;
            if (e == cudaSuccess && ms < best) { best = ms; bc = caps[ci]; bs = stg[si]; }
        }
    P.gemm_cap = bc;
    P.gemm_stages = bs;
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    if (best_ms) *best_ms = best;
    return e;
}

ccov_status group_status(GroupPlan& P, cudaStream_t st, const char* where) {
    P.sup.stream = st;
    return device_status(P.sup, where);
}

int64_t group_launches(const GroupPlan& P) { return P.launches; }
void group_shape(const GroupPlan& P, int* cap, int* stages) {
    int sms = 0, dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
    *cap = std::min(P.gemm_cap, sms);
    *stages = P.gemm_stages;
}

}  // namespace ccov
