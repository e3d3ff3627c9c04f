// Uncertainty from sub-reconstructions (Sec. 5): view graph, neighbourhoods
// grown from seed cameras, extraction of each sub-reconstruction, the
// covariances of all of them as one batch on the GPU, and the minimum-trace
// merge.  The planning and extraction are host work on the index set S; the
// covariances run in the library's kernels (grouped launches for the mixed
// form).  The rules are stated with the entry points in include/ccov.h.
#include <algorithm>
#include <cmath>
#include <cstring>
#include <limits>
#include <vector>

#include "ccov_internal.cuh"

namespace {

struct Edge {
    int to, w;
};

// Adjacency of the view graph, neighbours ascending, weight = shared points.
std::vector<std::vector<Edge>> view_graph(const ccov_obs* obs, int64_t t, int64_t n) {
    std::vector<uint64_t> keys;
    int64_t o = 0;
    while (o < t) {
        int64_t e = o;
        while (e < t && obs[e].pt == obs[o].pt) ++e;
        for (int64_t a = o; a < e; ++a)
            for (int64_t b = o; b < e; ++b)
                if (obs[a].cam != obs[b].cam) keys.push_back((uint64_t)obs[a].cam * (uint64_t)n + (uint64_t)obs[b].cam);
        o = e;
    }
    std::sort(keys.begin(), keys.end());
    std::vector<std::vector<Edge>> adj(n);
    for (size_t q = 0; q < keys.size();) {
        size_t r = q;
        while (r < keys.size() && keys[r] == keys[q]) ++r;
        adj[keys[q] / n].push_back({(int)(keys[q] % n), (int)(r - q)});
        q = r;
    }
    return adj;
}

// Best-first growth from `seed`: the camera of largest total weight to the
// chosen set (ties: the smaller index) until k cameras or none adjacent.
// score/chosen are n-sized scratch arrays, left as found.
std::vector<int> grow(int seed, int k, const std::vector<std::vector<Edge>>& adj, std::vector<int64_t>& score,
                      std::vector<char>& chosen) {
    std::vector<int> sel{seed}, touched;
    chosen[seed] = 1;
    for (const Edge& e : adj[seed]) {
        if (score[e.to] == 0) touched.push_back(e.to);
        score[e.to] += e.w;
    }
    while ((int)sel.size() < k) {
        int best = -1;
        int64_t best_s = 0;
        for (int c : touched) {
            if (chosen[c]) continue;
            if (score[c] > best_s || (score[c] == best_s && score[c] > 0 && c < best)) {
                best = c;
                best_s = score[c];
            }
        }
        if (best < 0) break;
        chosen[best] = 1;
        sel.push_back(best);
        for (const Edge& e : adj[best]) {
            if (chosen[e.to]) continue;
            if (score[e.to] == 0) touched.push_back(e.to);
            score[e.to] += e.w;
        }
    }
    for (int c : touched) score[c] = 0;
    for (int c : sel) chosen[c] = 0;
    std::sort(sel.begin(), sel.end());
    return sel;
}

ccov_status plan(const ccov_obs* obs, int64_t t, int64_t n, int64_t m, const ccov_subrecon_options* so,
                 std::vector<std::vector<int>>& subs) {
    if (!obs || !so || !so->seed_order || n < 1 || m < 1 || t < 1 || so->cams_per_sub < 2 || so->decompositions < 1)
        return CCOV_ERR_INVALID_ARG;
    for (int64_t o = 0; o < t; ++o) {
        if (obs[o].cam < 0 || obs[o].cam >= n || obs[o].pt < 0 || obs[o].pt >= m) return CCOV_ERR_INVALID_ARG;
        if (o > 0 && obs[o].pt < obs[o - 1].pt) return CCOV_ERR_INVALID_ARG;
    }
    for (int d = 0; d < so->decompositions; ++d) {
        std::vector<char> seen(n, 0);
        for (int64_t i = 0; i < n; ++i) {
            const int32_t c = so->seed_order[d * n + i];
            if (c < 0 || c >= n || seen[c]) return CCOV_ERR_INVALID_ARG;   // not a permutation
            seen[c] = 1;
        }
    }
    const auto adj = view_graph(obs, t, n);
    std::vector<int64_t> score(n, 0);
    std::vector<char> chosen(n, 0);
    for (int d = 0; d < so->decompositions; ++d) {
        std::vector<char> covered(n, 0);
        for (int64_t i = 0; i < n; ++i) {
            const int c = so->seed_order[d * n + i];
            if (covered[c]) continue;
            std::vector<int> S = grow(c, so->cams_per_sub, adj, score, chosen);
            for (int x : S) covered[x] = 1;
            subs.push_back(std::move(S));
        }
    }
    return CCOV_OK;
}

struct Sub {
    std::vector<int> cam_ids;   // global camera of each local camera
    std::vector<double> cams, pts, cov;
    std::vector<ccov_obs> obs;
};

// The sub-reconstruction of a camera set (pruned to >= 2 observations per
// camera and point), observations still sorted by point.
Sub extract(const double* cams, const double* pts, const ccov_obs* obs, const double* cov, int64_t t, int64_t n,
            int64_t m, const std::vector<int>& S) {
    std::vector<char> cam_in(n, 0), keep(t, 0);
    for (int c : S) cam_in[c] = 1;
    for (int64_t o = 0; o < t; ++o) keep[o] = cam_in[obs[o].cam];
    std::vector<int> cnt_pt(m), cnt_cam(n);
    while (true) {
        std::fill(cnt_pt.begin(), cnt_pt.end(), 0);
        for (int64_t o = 0; o < t; ++o)
            if (keep[o]) cnt_pt[obs[o].pt]++;
        for (int64_t o = 0; o < t; ++o)
            if (keep[o] && cnt_pt[obs[o].pt] < 2) keep[o] = 0;
        std::fill(cnt_cam.begin(), cnt_cam.end(), 0);
        for (int64_t o = 0; o < t; ++o)
            if (keep[o]) cnt_cam[obs[o].cam]++;
        bool dropped = false;
        for (int64_t o = 0; o < t; ++o)
            if (keep[o] && cnt_cam[obs[o].cam] < 2) { keep[o] = 0; dropped = true; }
        if (!dropped) break;
    }
    Sub sub;
    std::vector<int> cam_of(n, -1), pt_of(m, -1);
    for (int64_t o = 0; o < t; ++o)
        if (keep[o]) { cam_of[obs[o].cam] = 0; pt_of[obs[o].pt] = 0; }
    for (int64_t i = 0; i < n; ++i)
        if (cam_of[i] == 0) {
            cam_of[i] = (int)sub.cam_ids.size();
            sub.cam_ids.push_back((int)i);
            sub.cams.insert(sub.cams.end(), cams + 9 * i, cams + 9 * i + 9);
        }
    int np = 0;
    for (int64_t j = 0; j < m; ++j)
        if (pt_of[j] == 0) {
            pt_of[j] = np++;
            sub.pts.insert(sub.pts.end(), pts + 3 * j, pts + 3 * j + 3);
        }
    for (int64_t o = 0; o < t; ++o)
        if (keep[o]) {
            ccov_obs r = obs[o];
            r.cam = cam_of[r.cam];
            r.pt = pt_of[r.pt];
            sub.obs.push_back(r);
            if (cov) sub.cov.insert(sub.cov.end(), cov + 4 * o, cov + 4 * o + 4);
        }
    return sub;
}

}  // namespace

extern "C" {

ccov_status ccov_subrecon_plan(const ccov_obs* obs, int64_t t, int64_t n, int64_t m, const ccov_subrecon_options* sopt,
                               int64_t max_subs, int64_t max_total, int32_t* sub_ptr, int32_t* sub_cams,
                               int64_t* nsub, int64_t* total) {
    if (!nsub || !total) return CCOV_ERR_INVALID_ARG;
    std::vector<std::vector<int>> subs;
    ccov_status s = plan(obs, t, n, m, sopt, subs);
    if (s != CCOV_OK) return s;
    int64_t tot = 0;
    for (const auto& S : subs) tot += (int64_t)S.size();
    *nsub = (int64_t)subs.size();
    *total = tot;
    if (max_subs < (int64_t)subs.size() || max_total < tot || !sub_ptr || !sub_cams) return CCOV_ERR_INVALID_ARG;
    int64_t off = 0;
    for (size_t q = 0; q < subs.size(); ++q) {
        sub_ptr[q] = (int32_t)off;
        for (int c : subs[q]) sub_cams[off++] = c;
    }
    sub_ptr[subs.size()] = (int32_t)off;
    return CCOV_OK;
}

ccov_status ccov_subrecon_covariance(const double* cameras, int64_t n, const double* points, int64_t m,
                                     const ccov_obs* obs, int64_t t, double sigma, const double* obs_cov,
                                     const ccov_options* opt, const ccov_subrecon_options* sopt, double* out,
                                     int32_t* cover, int64_t* nsub) {
    if (!cameras || !points || !out) return CCOV_ERR_INVALID_ARG;
    if (opt && opt->input_memory == CCOV_MEM_DEVICE) return CCOV_ERR_INVALID_ARG;   // host inputs only
    std::vector<std::vector<int>> subs;
    ccov_status s = plan(obs, t, n, m, sopt, subs);
    if (s != CCOV_OK) return s;
    // sub-reconstructions, each as a context of its own
    std::vector<Sub> parts;
    std::vector<ccov_ctx*> ctxs;
    for (const auto& S : subs) {
        Sub sub = extract(cameras, points, obs, obs_cov, t, n, m, S);
        if (sub.cam_ids.size() < 2) continue;
        ccov_ctx* h = nullptr;
        ccov_status cs = ccov_create(sub.cams.data(), (int64_t)sub.cam_ids.size(), sub.pts.data(),
                                     (int64_t)sub.pts.size() / 3, sub.obs.data(), (int64_t)sub.obs.size(), sigma,
                                     obs_cov ? sub.cov.data() : nullptr, opt, nullptr, &h);
        if (cs != CCOV_OK) {          // a degenerate neighbourhood is skipped
            ccov_destroy(h);
            if (cs == CCOV_ERR_DEGENERATE || cs == CCOV_ERR_INVALID_ARG) continue;
            for (ccov_ctx* x : ctxs) ccov_destroy(x);
            return cs;
        }
        ctxs.push_back(h);
        parts.push_back(std::move(sub));
    }
    const int k = (int)ctxs.size();
    std::vector<int64_t> off(k + 1, 0);
    for (int q = 0; q < k; ++q) off[q + 1] = off[q] + 81 * (int64_t)parts[q].cam_ids.size();
    double* d_out = nullptr;
    std::vector<double*> outs(k);
    std::vector<char> ok(k, 1);
    if (k > 0) {
        if (cudaMalloc(&d_out, sizeof(double) * off[k]) != cudaSuccess) {
            for (ccov_ctx* x : ctxs) ccov_destroy(x);
            return CCOV_ERR_OOM;
        }
        for (int q = 0; q < k; ++q) outs[q] = d_out + off[q];
        ccov_batch* b = nullptr;
        ccov_status bs = ccov_batch_create_ex(ctxs.data(), k, outs.data(), CCOV_BATCH_AUTO | CCOV_BATCH_NO_TUNE, &b);
        if (bs == CCOV_OK) {
            bs = ccov_batch_run(b, nullptr);
            ccov_batch_destroy(b);
        }
        if (bs != CCOV_OK) {
            // some sub-reconstruction failed on the device: solve one by one and skip the failures
            for (int q = 0; q < k; ++q) {
                ccov_ctx* h = ctxs[q];
                ccov_status r = ccov_information(h);
                if (r == CCOV_OK) r = ccov_schur(h);
                if (r == CCOV_OK) r = ccov_nullspace(h, nullptr);
                if (r == CCOV_OK) r = ccov_covariance(h, outs[q], CCOV_MEM_DEVICE, nullptr);
                ok[q] = r == CCOV_OK;
            }
        }
    }
    std::vector<double> host(off[k]);
    if (k > 0 && cudaMemcpy(host.data(), d_out, sizeof(double) * off[k], cudaMemcpyDeviceToHost) != cudaSuccess) {
        cudaFree(d_out);
        for (ccov_ctx* x : ctxs) ccov_destroy(x);
        return CCOV_ERR_CUDA;
    }
    if (d_out) cudaFree(d_out);
    for (ccov_ctx* x : ctxs) ccov_destroy(x);
    // minimum-trace merge
    std::vector<double> best(n, std::numeric_limits<double>::infinity());
    for (int64_t e = 0; e < 81 * n; ++e) out[e] = std::numeric_limits<double>::quiet_NaN();
    if (cover) std::fill(cover, cover + n, 0);
    int64_t solved = 0;
    for (int q = 0; q < k; ++q) {
        if (!ok[q]) continue;
        ++solved;
        for (size_t a = 0; a < parts[q].cam_ids.size(); ++a) {
            const double* blk = host.data() + off[q] + 81 * a;
            const int c = parts[q].cam_ids[a];
            double tr = 0.0;
            for (int d = 0; d < 9; ++d) tr += blk[10 * d];
            if (cover) cover[c]++;
            if (tr < best[c]) {
                best[c] = tr;
                std::memcpy(out + 81 * (int64_t)c, blk, sizeof(double) * 81);
            }
        }
    }
    if (nsub) *nsub = solved;
    return CCOV_OK;
}

}  // extern "C"
