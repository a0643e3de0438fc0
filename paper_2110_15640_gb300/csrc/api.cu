// api.cu -- the C ABI of libgcmc (declared in include/gcmc.h): contexts, validated uploads, the
// per-run workspace, S1 grouping, plain / batched / asynchronous runs, debug outputs, post-scale.
#include <algorithm>
#include <chrono>
#include <cmath>
#include <cstdio>
#include <cstring>
#include <deque>
#include <map>
#include <string>
#include <thread>
#include <vector>

#include "internal.h"

using namespace gcmc;

namespace {

struct GridH {
    DevGrid dg{};
    std::vector<double> r, lat, lon;
    std::vector<void *> owned;
};

struct OpacH {
    int kind = 0, grid = -1, nlam = 0;
    AlbDev alb{};
    KtabDev kt{};
    XsecDev xs{};
    std::vector<double> lam;          // band centres (k-table) or table wavelengths (xsec)
    std::vector<void *> owned;
};

struct Ticket {
    cudaEvent_t done = nullptr;
    int n_jobs = 0;
    unsigned long long *h_acc = nullptr;   // pinned [n_jobs][ACC_SLOTS]
    double *h_info = nullptr;              // pinned [n_jobs][4]: L_tot, n_incl, cdf_total, mode
    void *ws = nullptr;                    // this ticket's workspace
};

}  // namespace

struct gcmc_ctx {
    int device = 0;
    cudaStream_t stream = nullptr;
    gcmc_alloc_fn alloc = nullptr;
    gcmc_free_fn free_fn = nullptr;
    void *user = nullptr;
    std::vector<GridH> grids;
    std::vector<OpacH> opacs;
    std::vector<gcmc_source_desc> sources;
    DevGrid *d_grids = nullptr;
    int grid_cap = 256;
    void *arena = nullptr;
    size_t arena_n = 0;
    unsigned long long *h_acc = nullptr;   // pinned readback staging
    double *h_info = nullptr;
    size_t h_cap = 0;
    std::map<uint64_t, Ticket> tickets;
    uint64_t next_ticket = 1;
    std::string err;
    struct Staging {
        char *ptr = nullptr;
        size_t cap = 0;
        cudaEvent_t ev = nullptr;
    } stg[2];                              // pinned staging of job records, used in turn
    int stg_i = 0;
    bool prof = false;                     // profiling: events around S1 and transport of each run
    std::vector<cudaEvent_t> prof_ev;      // triples (before S1, before transport, after transport)
};

namespace {

gcmc_status fail(gcmc_ctx *c, gcmc_status s, const std::string &m)
{
    if (c) c->err = m;
    return s;
}

gcmc_status cuda_fail(gcmc_ctx *c, cudaError_t e, const char *where)
{
    return fail(c, GCMC_ERR_CUDA, std::string(where) + ": " + cudaGetErrorString(e));
}

#define CK(call)                                                   \
    do {                                                           \
        cudaError_t e_ = (call);                                   \
        if (e_ != cudaSuccess) return cuda_fail(ctx, e_, #call);   \
    } while (0)

void *dalloc(gcmc_ctx *ctx, size_t bytes)
{
    if (bytes == 0) bytes = 256;
    if (ctx->alloc) return ctx->alloc(bytes, ctx->user);
    void *p = nullptr;
    if (cudaMalloc(&p, bytes) != cudaSuccess) return nullptr;
    return p;
}

void dfree(gcmc_ctx *ctx, void *p)
{
    if (!p) return;
    if (ctx->free_fn) ctx->free_fn(p, ctx->user);
    else cudaFree(p);
}

template <typename T> T *dput(gcmc_ctx *ctx, std::vector<void *> &owned, const T *src, size_t n, cudaError_t &e)
{
    T *d = (T *)dalloc(ctx, n * sizeof(T));
    if (!d) {
        e = cudaErrorMemoryAllocation;
        return nullptr;
    }
    owned.push_back(d);
    if (src && n) {
        const cudaError_t r = cudaMemcpyAsync(d, src, n * sizeof(T), cudaMemcpyDefault, ctx->stream);
        if (r != cudaSuccess) e = r;
    }
    return d;
}

template <typename T> bool fetch(gcmc_ctx *ctx, const T *src, size_t n, int memory, std::vector<T> &out)
{
    out.resize(n);
    if (!src) return false;
    if (!n) return true;
    if (memory == GCMC_MEM_DEVICE) {
        if (cudaMemcpyAsync(out.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost, ctx->stream) != cudaSuccess)
            return false;
        return cudaStreamSynchronize(ctx->stream) == cudaSuccess;
    }
    std::memcpy(out.data(), src, n * sizeof(T));
    return true;
}

bool strictly_increasing(const std::vector<double> &v)
{
    for (size_t i = 0; i + 1 < v.size(); ++i)
        if (!(v[i + 1] > v[i])) return false;
    for (double x : v)
        if (!std::isfinite(x)) return false;
    return true;
}

void perp_basis(const double s[3], double e1[3], double e2[3])
{
    double a[3] = {0.0, 0.0, 1.0};
    if (std::fabs(s[2]) >= 0.9) {
        a[0] = 1.0;
        a[2] = 0.0;
    }
    e1[0] = s[1] * a[2] - s[2] * a[1];
    e1[1] = s[2] * a[0] - s[0] * a[2];
    e1[2] = s[0] * a[1] - s[1] * a[0];
    const double n = std::sqrt(e1[0] * e1[0] + e1[1] * e1[1] + e1[2] * e1[2]);
    for (int i = 0; i < 3; ++i) e1[i] /= n;
    e2[0] = s[1] * e1[2] - s[2] * e1[1];
    e2[1] = s[2] * e1[0] - s[0] * e1[2];
    e2[2] = s[0] * e1[1] - s[1] * e1[0];
}

size_t align256(size_t x) { return (x + 255) & ~(size_t)255; }


// ------------------------------------------------------------------ run planning
struct Group {
    int grid, opac, mode, precision, source;
    std::vector<int> members;
    int nprep = 0;                      // cell-table preparations (a band job has one per g-ordinate)
};

struct Plan {
    std::vector<DevJob> jobs;
    std::vector<PrepJob> prep;          // in group order (members of a group are contiguous)
    std::vector<int> prep_pos;          // position of job q in `prep`
    std::vector<int> job_group;         // group of job q
    std::vector<Group> groups;
    std::vector<size_t> off_rec, off_alpha, off_cdf, off_w, off_info, off_bsum, off_bcnt;
    std::vector<int> ng_s;              // g-ordinates a band job samples (0: one g-ordinate)
    std::vector<int64_t> nblk;          // emission scan blocks per preparation
    std::vector<size_t> g_first;
    size_t off_jobs = 0, off_prep = 0, off_acc = 0, off_work = 0, off_gather = 0, ws_bytes = 0;
    int64_t total_items = 0;
    bool scatter = false;               // some job follows scattered packets (albedo)
    int feat = 0;                       // optional kernel code the jobs need (FEAT_BAND, FEAT_EXT)
    int one_grid = 1;                   // every job uses the same grid
    int tab_n = 0;                      // largest march-table size (pair entries) of the jobs' grids
};

// FP32 cross-section jobs: the table wavelengths that bracket every Doppler-shifted wavelength of the
// grid, lambda_0 (1 + d) for d in [dmin, dmax], as FP32 offsets lambda_l / lambda_0 - 1 (xs_n = -1 when
// the window reaches a table edge or is longer than XS_LOCAL: the kernel then brackets in FP64)
void xsec_window(const OpacH &o, PrepJob &pj)
{
    const std::vector<double> &lam = o.lam;
    const double a = pj.lam_m * (1.0 + o.xs.dmin), b = pj.lam_m * (1.0 + o.xs.dmax);
    pj.xs_lo = 0;
    pj.xs_n = -1;
    if (!(a > lam.front() && b < lam.back())) return;
    const int lo = (int)(std::upper_bound(lam.begin(), lam.end(), a) - lam.begin()) - 1;   // last lam <= a
    const int hi = (int)(std::upper_bound(lam.begin(), lam.end(), b) - lam.begin());       // first lam > b
    const int n = hi - lo + 1;
    if (lo < 0 || n > XS_LOCAL) return;
    for (int t = 0; t < n; ++t) pj.xs_d[t] = (float)((lam[lo + t] - pj.lam_m) / pj.lam_m);
    pj.xs_lo = lo;
    pj.xs_n = n;
}

gcmc_status check_job(gcmc_ctx *ctx, const gcmc_job &j)
{
    if (j.grid_id < 0 || j.grid_id >= (int)ctx->grids.size()) return fail(ctx, GCMC_ERR_ARG, "bad grid_id");
    if (j.opac_id < 0 || j.opac_id >= (int)ctx->opacs.size()) return fail(ctx, GCMC_ERR_ARG, "bad opac_id");
    if (j.source_id < 0 || j.source_id >= (int)ctx->sources.size()) return fail(ctx, GCMC_ERR_ARG, "bad source_id");
    const OpacH &o = ctx->opacs[j.opac_id];
    if (!ctx->grids[j.grid_id].dg.r) return fail(ctx, GCMC_ERR_ARG, "grid was released");
    if (o.grid != j.grid_id) return fail(ctx, GCMC_ERR_ARG, "opacity released or belongs to another grid");
    if (j.mode < 0 || j.mode > 2) return fail(ctx, GCMC_ERR_ARG, "bad mode");
    const int want = j.mode == GCMC_ALBEDO ? GCMC_OPAC_ALBEDO : j.mode == GCMC_EMISSION ? GCMC_OPAC_KTABLE : GCMC_OPAC_XSEC;
    // transmission runs on cross-sections (chords) or on scattering opacities (chords, optionally
    // followed by multiple scattering)
    // emission runs on k-tables or on cross-sections (high resolution, Doppler-shifted)
    const bool kind_ok = o.kind == want || (j.mode == GCMC_TRANSMISSION && o.kind == GCMC_OPAC_ALBEDO) ||
                         (j.mode == GCMC_EMISSION && o.kind == GCMC_OPAC_XSEC);
    if (!kind_ok) return fail(ctx, GCMC_ERR_ARG, "opacity kind does not match the mode");
    if (j.n_packets < 0) return fail(ctx, GCMC_ERR_ARG, "negative n_packets");
    const gcmc_source_desc &s = ctx->sources[j.source_id];
    if (j.obs_idx >= s.n_obs) return fail(ctx, GCMC_ERR_ARG, "obs_idx out of range");
    if (j.mode == GCMC_EMISSION && s.scatter_emission)
        return fail(ctx, GCMC_ERR_ARG, "scattering after emission needs scattering opacities (not in k-tables)");
    if (j.mode == GCMC_TRANSMISSION && s.trans_scatter && o.kind != GCMC_OPAC_ALBEDO)
        return fail(ctx, GCMC_ERR_ARG, "multiple scattering in transmission needs scattering opacities");
    if (o.kind == GCMC_OPAC_ALBEDO || o.kind == GCMC_OPAC_XSEC) {
        if (j.lam_idx < 0 || j.lam_idx >= o.nlam) return fail(ctx, GCMC_ERR_ARG, "lam_idx out of range");
    } else if (j.lam_idx < 0 || j.lam_idx >= o.kt.nb || j.g_idx < -1 || j.g_idx >= o.kt.ng) {
        return fail(ctx, GCMC_ERR_ARG, "band / g index out of range");
    } else if (j.g_idx == -1 && !o.kt.gw) {
        return fail(ctx, GCMC_ERR_ARG, "a band job (g_idx = -1) needs the k-table's g weights");
    }
    return GCMC_OK;
}

// the tally columns of a checked job: observers (one when obs_idx >= 0), or the transit columns
static int job_columns(const gcmc_ctx *ctx, const gcmc_job &j)
{
    const gcmc_source_desc &s = ctx->sources[j.source_id];
    if (j.mode == GCMC_TRANSMISSION) return s.trans_scatter ? 2 : 1;
    return j.obs_idx >= 0 ? 1 : s.n_obs;
}

gcmc_status plan_run(gcmc_ctx *ctx, const gcmc_job *jobs, int n, int chunk, Plan &P)
{
    if (n <= 0 || !jobs) return fail(ctx, GCMC_ERR_ARG, "no jobs");
    if (chunk <= 0 || chunk % 32) return fail(ctx, GCMC_ERR_ARG, "chunk must be a positive multiple of 32");
    for (int q = 0; q < n; ++q) {
        const gcmc_status s = check_job(ctx, jobs[q]);
        if (s) return s;
    }
    P.jobs.resize(n);
    P.prep_pos.resize(n);
    P.job_group.assign(n, 0);
    P.off_rec.assign(n, 0);
    P.off_alpha.assign(n, 0);
    P.off_cdf.assign(n, 0);
    P.off_w.assign(n, 0);
    P.off_info.assign(n, 0);
    P.off_bsum.assign(n, 0);
    P.off_bcnt.assign(n, 0);
    P.ng_s.assign(n, 0);
    P.nblk.assign(n, 0);
    for (int q = 0; q < n; ++q) {
        const gcmc_job &j = jobs[q];
        const gcmc_source_desc &s = ctx->sources[j.source_id];
        if (j.mode == GCMC_EMISSION && j.g_idx < 0) P.ng_s[q] = ctx->opacs[j.opac_id].kt.ng;
        const int prec = s.precision == GCMC_FP64 ? GCMC_FP64 : GCMC_FP32;
        int gi = -1;
        for (size_t g = 0; g < P.groups.size(); ++g) {
            const Group &G = P.groups[g];
            if (G.grid == j.grid_id && G.opac == j.opac_id && G.mode == j.mode && G.precision == prec &&
                (j.mode != GCMC_EMISSION || G.source == j.source_id))
                gi = (int)g;
        }
        if (gi < 0) {
            P.groups.push_back({j.grid_id, j.opac_id, j.mode, prec, j.source_id, {}});
            gi = (int)P.groups.size() - 1;
        }
        P.groups[gi].members.push_back(q);
        P.groups[gi].nprep += std::max(1, P.ng_s[q]);
        P.job_group[q] = gi;
    }
    size_t ws = 0, n_prep = 0;
    for (int q = 0; q < n; ++q) {
        const gcmc_job &j = jobs[q];
        const int prec = ctx->sources[j.source_id].precision == GCMC_FP64 ? GCMC_FP64 : GCMC_FP32;
        const int64_t ncell = ctx->grids[j.grid_id].dg.ncell;
        const size_t esz = prec == GCMC_FP64 ? 8 : 4;
        const int m = std::max(1, P.ng_s[q]);     // tables per job: one per g-ordinate of a band job
        n_prep += m;
        P.off_rec[q] = ws;
        ws += align256((size_t)m * ncell * (ctx->opacs[j.opac_id].kind == GCMC_OPAC_ALBEDO ? 4 * esz : esz));
        if (ctx->opacs[j.opac_id].kind == GCMC_OPAC_ALBEDO) {   // compact alpha beside the records
            P.off_alpha[q] = ws;
            ws += align256((size_t)ncell * esz);
        }
        if (j.mode == GCMC_EMISSION) {
            const int64_t nblk = std::max<int64_t>((ncell + EMIS_SCAN_BLOCK - 1) / EMIS_SCAN_BLOCK,
                                                   emis_col_blocks(ctx->grids[j.grid_id].dg));
            P.nblk[q] = nblk;
            P.off_cdf[q] = ws;
            ws += align256((size_t)m * ncell * 8);
            P.off_w[q] = ws;
            ws += align256((size_t)m * ncell * esz);
            P.off_info[q] = ws;
            // band job: summary info block, the g table, then one info block per g-ordinate
            ws += P.ng_s[q] ? 256 + align256((size_t)m * GTAB_ROW * 8) + (size_t)m * GINFO_STRIDE * 8 : 256;
            P.off_bsum[q] = ws;
            ws += align256((size_t)m * nblk * 8);
            P.off_bcnt[q] = ws;
            ws += align256((size_t)m * nblk * 8);
        }
    }
    const size_t ng = P.groups.size();
    P.g_first.resize(ng);
    P.off_jobs = ws;
    ws += align256(n * sizeof(DevJob));
    P.off_prep = ws;
    ws += align256(n_prep * sizeof(PrepJob));
    P.off_acc = ws;
    ws += align256((size_t)n * ACC_SLOTS * 8);
    P.off_work = ws;
    ws += 256;
    P.off_gather = ws;
    ws += align256((size_t)n * 4 * sizeof(double));
    P.ws_bytes = ws;

    int64_t items = 0;
    P.prep.clear();
    for (size_t g = 0; g < ng; ++g) {
        P.g_first[g] = P.prep.size();
        for (int q : P.groups[g].members) {
            P.prep_pos[q] = (int)P.prep.size();
            PrepJob pj;
            std::memset(&pj, 0, sizeof(pj));
            const gcmc_job &j = jobs[q];
            const OpacH &o = ctx->opacs[j.opac_id];
            pj.lam = j.lam_idx;
            pj.g = j.g_idx;
            pj.lam_hint = j.lam_idx;
            if (o.kind == GCMC_OPAC_KTABLE) {
                pj.lam_m = o.lam[j.lam_idx];
            } else if (o.kind == GCMC_OPAC_XSEC) {
                pj.lam_m = o.lam[j.lam_idx];
                xsec_window(o, pj);
            }
            if (P.ng_s[q]) {
                // a band job: the tables of every g-ordinate, prepared like ng single jobs
                for (int gi = 0; gi < P.ng_s[q]; ++gi) {
                    pj.g = gi;
                    P.prep.push_back(pj);
                }
            } else {
                P.prep.push_back(pj);
            }
        }
    }
    for (int q = 0; q < n; ++q) {
        const gcmc_job &j = jobs[q];
        const gcmc_source_desc &s = ctx->sources[j.source_id];
        DevJob &d = P.jobs[q];
        std::memset(&d, 0, sizeof(d));
        d.mode = j.mode;
        d.rec4 = ctx->opacs[j.opac_id].kind == GCMC_OPAC_ALBEDO;
        if (d.rec4) P.scatter = true;
        d.grid_slot = j.grid_id;
        d.survival = s.survival;
        d.precision = s.precision == GCMC_FP64 ? GCMC_FP64 : GCMC_FP32;
        d.key = j.job_key;
        d.seed = j.seed;
        d.n_packets = j.n_packets;
        d.max_steps = s.max_steps > 0 ? s.max_steps : ((int64_t)1 << 40);
        for (int a = 0; a < 3; ++a) d.star[a] = s.star[a];
        perp_basis(d.star, d.e1, d.e2);
        if (j.obs_idx >= 0) {
            d.n_obs = 1;
            for (int a = 0; a < 3; ++a) d.obs[0][a] = s.obs[j.obs_idx][a];
        } else {
            d.n_obs = j.mode == GCMC_TRANSMISSION ? 1 : s.n_obs;
            for (int o = 0; o < d.n_obs; ++o)
                for (int a = 0; a < 3; ++a) d.obs[o][a] = s.obs[o][a];
        }
        if (j.mode == GCMC_TRANSMISSION) {
            // the transit observer looks along the chords, -star
            d.n_obs = 1;
            for (int a = 0; a < 3; ++a) d.obs[0][a] = -s.star[a];
            d.trans_scatter = s.trans_scatter ? 1 : 0;
            d.ld_law = s.ld_law;
            for (int c = 0; c < 4; ++c) d.ld_c[c] = s.ld_coef[c];
            d.star_r = s.star_radius;
            d.tr_x = s.transit_xy[0];
            d.tr_y = s.transit_xy[1];
        }
        d.n_tal = job_columns(ctx, j);
        d.forced_first = s.forced_first;
        d.path_bias = s.path_bias;
        d.cont_abs = s.cont_abs && d.rec4 ? 1 : 0;   // needs the scattering records' omega
        if (s.surface_albedo > 0.0 || s.cloud_phase == GCMC_CLOUD_TTHG || (j.mode == GCMC_TRANSMISSION &&
            (s.trans_scatter || s.ld_law != GCMC_LD_NONE)) || d.forced_first || d.cont_abs)
            P.feat |= FEAT_EXT;
        if (d.cont_abs) P.feat |= FEAT_EXT | FEAT_CABS;
        d.ng_s = P.ng_s[q];
        if (d.ng_s) {
            P.feat |= FEAT_BAND;
            d.g_bias = s.g_bias;
            d.g_beta = s.g_beta;
            d.gw = ctx->opacs[j.opac_id].kt.gw;
        }
        for (int c = 0; c < 4; ++c) d.ld_c_f[c] = (float)d.ld_c[c];
        d.star_r_f = (float)d.star_r;
        d.tr_x_f = (float)d.tr_x;
        d.tr_y_f = (float)d.tr_y;
        d.w_rr = s.w_rr;
        d.p_surv = s.p_surv;
        d.tau_cut = s.tau_peel_cut;
        d.hg_eps = s.hg_iso_eps;
        d.cloud_phase = s.cloud_phase;
        d.surf_as = s.surface_albedo;
        d.surf_as_f = (float)s.surface_albedo;
        for (int a = 0; a < 3; ++a) {
            d.star_f[a] = (float)d.star[a];
            d.e1_f[a] = (float)d.e1[a];
            d.e2_f[a] = (float)d.e2[a];
        }
        for (int o = 0; o < MAX_OBS; ++o)
            for (int a = 0; a < 3; ++a) d.obs_f[o][a] = (float)d.obs[o][a];
        d.w_rr_f = (float)d.w_rr;
        d.p_surv_f = (float)d.p_surv;
        d.hg_eps_f = (float)d.hg_eps;
        d.chunk_begin = items;
        items += (j.n_packets + chunk - 1) / chunk;
    }
    P.total_items = items;
    for (int q = 0; q < n; ++q) {
        const DevGrid &g = ctx->grids[jobs[q].grid_id].dg;
        P.tab_n = std::max(P.tab_n, tab_entries(g.nlon, g.nlat, g.nr));
        if (jobs[q].grid_id != jobs[0].grid_id) P.one_grid = 0;
    }
    return GCMC_OK;
}

// a band job's g-sampling table (Sect. 4.7) from its g-ordinates' luminosities:
// p(g) = w_g L_g / sum w L, q(g) by the source's bias, W_g = p / q; summary info L_band = sum w L
__device__ void band_table(DevJob &J)
{
    const int ng = J.ng_s;
    double sum = 0.0, ninc = 0.0;
    for (int g = 0; g < ng; ++g) {
        const double *inf = J.ginfo + (size_t)g * GINFO_STRIDE;
        const double wl = J.gw[g] * inf[INFO_LTOT];
        J.gtab[g * GTAB_ROW + 2] = wl;
        sum += wl;
        ninc += inf[INFO_NINCL];
    }
    double cum = 0.0;
    for (int g = 0; g < ng; ++g) {
        const double p = sum > 0.0 ? J.gtab[g * GTAB_ROW + 2] / sum : 0.0;
        const double qg = J.g_bias == GCMC_GBIAS_UNIFORM     ? 1.0 / ng
                          : J.g_bias == GCMC_GBIAS_COMPOSITE ? (1.0 - J.g_beta) * p + J.g_beta / ng
                                                              : p;
        cum += qg;
        J.gtab[g * GTAB_ROW] = cum;
        J.gtab[g * GTAB_ROW + 1] = qg > 0.0 ? p / qg : 0.0;
        reinterpret_cast<long long *>(J.gtab)[g * GTAB_ROW + 3] =
            reinterpret_cast<const long long *>(J.ginfo + (size_t)g * GINFO_STRIDE)[INFO_QTOT];
    }
    double *summary = const_cast<double *>(J.info);   // the band job's own summary block in its workspace
    summary[INFO_LTOT] = sum;
    summary[INFO_NINCL] = ninc;
    summary[INFO_CDFTOT] = cum;
}

__global__ void k_finalize_jobs(DevJob *jobs, int n)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    if (jobs[q].mode == GCMC_EMISSION && jobs[q].ng_s > 0) {
        band_table(jobs[q]);
    } else if (jobs[q].mode == GCMC_EMISSION) {
        const long long qtot = reinterpret_cast<const long long *>(jobs[q].info)[INFO_QTOT];
        jobs[q].cdf_step_fix = jobs[q].n_packets > 0 ? qtot / jobs[q].n_packets : 0;
    }
}

// S1 for every job of the plan, then the device job array, accumulators and work counter.
// Host staging of the job records: copies from pinned memory are asynchronous, whereas a copy from
// pageable memory synchronises the stream first.  The context keeps two pinned buffers and uses them
// in turn, each guarded by an event after its copies; callers with their own pinned slot (the
// server, one per job slot) pass it as host_stage.
char *stage_buffer(gcmc_ctx *ctx, size_t bytes, cudaEvent_t *ev_out)
{
    gcmc_ctx::Staging &b = ctx->stg[ctx->stg_i ^= 1];
    if (b.ev) cudaEventSynchronize(b.ev);
    else if (cudaEventCreateWithFlags(&b.ev, cudaEventDisableTiming) != cudaSuccess) return nullptr;
    if (b.cap < bytes) {
        if (b.ptr) cudaFreeHost(b.ptr);
        b.ptr = nullptr;
        b.cap = 0;
        if (cudaMallocHost((void **)&b.ptr, bytes) != cudaSuccess) return nullptr;
        b.cap = bytes;
    }
    *ev_out = b.ev;
    return b.ptr;
}

gcmc_status stage(gcmc_ctx *ctx, Plan &P, char *base, double *lum = nullptr, char *host_stage = nullptr)
{
    const int n = (int)P.jobs.size();
    for (int q = 0; q < n; ++q) {
        DevJob &d = P.jobs[q];
        const int m = std::max(1, P.ng_s[q]);
        const size_t ncell = (size_t)ctx->grids[P.groups[P.job_group[q]].grid].dg.ncell;
        const size_t esz = d.precision == GCMC_FP64 ? 8 : 4;
        d.acc = reinterpret_cast<unsigned long long *>(base + P.off_acc) + (size_t)q * ACC_SLOTS;
        for (int gi = 0; gi < m; ++gi) {
            PrepJob &pj = P.prep[P.prep_pos[q] + gi];
            pj.rec = base + P.off_rec[q] + gi * ncell * esz;
            pj.alpha = d.rec4 ? base + P.off_alpha[q] : nullptr;
            if (d.mode == GCMC_EMISSION) {
                pj.cdf = reinterpret_cast<long long *>(base + P.off_cdf[q]) + gi * ncell;
                pj.wcell = base + P.off_w[q] + gi * ncell * esz;
                pj.info = reinterpret_cast<double *>(base + P.off_info[q]) +
                          (P.ng_s[q] ? (256 + align256((size_t)m * GTAB_ROW * 8)) / 8 + (size_t)gi * GINFO_STRIDE : 0);
                pj.bsum = reinterpret_cast<double *>(base + P.off_bsum[q]) + gi * P.nblk[q];
                pj.bcnt = reinterpret_cast<double *>(base + P.off_bcnt[q]) + gi * P.nblk[q];
                pj.lum = P.ng_s[q] ? nullptr : lum;
            }
        }
        const PrepJob &p0 = P.prep[P.prep_pos[q]];
        d.rec = p0.rec;
        d.arec = p0.alpha;
        if (d.mode == GCMC_EMISSION) {
            d.cdf = p0.cdf;
            d.wcell = p0.wcell;
            d.info = reinterpret_cast<double *>(base + P.off_info[q]);   // a band job's summary block
            if (P.ng_s[q]) {
                d.gtab = reinterpret_cast<double *>(base + P.off_info[q] + 256);
                d.ginfo = p0.info;
            }
        }
    }
    PrepJob *dprep = reinterpret_cast<PrepJob *>(base + P.off_prep);
    DevJob *djobs = reinterpret_cast<DevJob *>(base + P.off_jobs);
    const size_t bp = P.prep.size() * sizeof(PrepJob), bj = n * sizeof(DevJob);
    cudaEvent_t stg_ev = nullptr;
    char *hs = host_stage ? host_stage : stage_buffer(ctx, bp + bj, &stg_ev);
    if (!hs) return fail(ctx, GCMC_ERR_OOM, "pinned staging");
    std::memcpy(hs, P.prep.data(), bp);
    std::memcpy(hs + bp, P.jobs.data(), bj);
    CK(cudaMemcpyAsync(dprep, hs, bp, cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaMemcpyAsync(djobs, hs + bp, bj, cudaMemcpyHostToDevice, ctx->stream));
    if (stg_ev) CK(cudaEventRecord(stg_ev, ctx->stream));
    for (size_t g = 0; g < P.groups.size(); ++g) {
        const Group &G = P.groups[g];
        const PrepJob *gp = dprep + P.g_first[g];
        const int m = G.nprep;
        const GridH &gh = ctx->grids[G.grid];
        const OpacH &oh = ctx->opacs[G.opac];
        cudaError_t e;
        if (oh.kind == GCMC_OPAC_ALBEDO) {
            e = prep_albedo(G.precision, ctx->d_grids + G.grid, gh.dg, oh.alb, gp, m, ctx->stream);
        } else if (oh.kind == GCMC_OPAC_KTABLE) {
            const gcmc_source_desc &s = ctx->sources[G.source];
            e = prep_emission(G.precision, gh.dg, oh.kt, gp, m, s.tau_vert_max, s.beta_emis, ctx->stream);
        } else if (G.mode == GCMC_EMISSION) {
            const gcmc_source_desc &s = ctx->sources[G.source];
            e = prep_emission_xsec(G.precision, gh.dg, oh.xs, gp, m, s.tau_vert_max, s.beta_emis, ctx->stream);
        } else {
            e = prep_xsec(G.precision, gh.dg, oh.xs, gp, m, ctx->stream);
        }
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cell-table kernels");
    }
    count_launch(1);
    k_finalize_jobs<<<(n + 127) / 128, 128, 0, ctx->stream>>>(djobs, n);
    CK(cudaGetLastError());
    CK(cudaMemsetAsync(base + P.off_acc, 0, (size_t)n * ACC_SLOTS * 8, ctx->stream));
    CK(cudaMemsetAsync(base + P.off_work, 0, 256, ctx->stream));
    return GCMC_OK;
}

void prof_mark(gcmc_ctx *ctx)
{
    if (!ctx->prof) return;
    cudaEvent_t e;
    if (cudaEventCreate(&e) == cudaSuccess) {
        cudaEventRecord(e, ctx->stream);
        ctx->prof_ev.push_back(e);
    }
}

gcmc_status ensure_arena(gcmc_ctx *ctx, size_t bytes)
{
    if (ctx->arena_n >= bytes) return GCMC_OK;
    if (ctx->arena) {
        cudaStreamSynchronize(ctx->stream);
        dfree(ctx, ctx->arena);
        ctx->arena = nullptr;
        ctx->arena_n = 0;
    }
    const size_t want = bytes + bytes / 8;
    ctx->arena = dalloc(ctx, want);
    if (!ctx->arena) return fail(ctx, GCMC_ERR_OOM, "workspace allocation failed");
    ctx->arena_n = want;
    return GCMC_OK;
}

gcmc_status ensure_host(gcmc_ctx *ctx, size_t njobs)
{
    if (ctx->h_cap >= njobs) return GCMC_OK;
    if (ctx->h_acc) cudaFreeHost(ctx->h_acc);
    if (ctx->h_info) cudaFreeHost(ctx->h_info);
    ctx->h_acc = nullptr;
    ctx->h_info = nullptr;
    CK(cudaMallocHost((void **)&ctx->h_acc, njobs * ACC_SLOTS * 8));
    CK(cudaMallocHost((void **)&ctx->h_info, njobs * 4 * sizeof(double)));
    ctx->h_cap = njobs;
    return GCMC_OK;
}

__global__ void k_gather_info(const DevJob *jobs, int n, double *out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n) return;
    if (jobs[q].mode == GCMC_EMISSION) {
        out[4 * q] = jobs[q].info[0];
        out[4 * q + 1] = jobs[q].info[1];
        out[4 * q + 2] = jobs[q].info[2];
    } else {
        out[4 * q] = out[4 * q + 1] = out[4 * q + 2] = 0.0;
    }
    out[4 * q + 3] = (double)jobs[q].mode;
}

// convert one job's accumulators into tallies and stats
void unpack(const unsigned long long *acc, const double *info, int n_obs, double *tally, gcmc_stats *st)
{
    for (int o = 0; o < MAX_OBS; ++o) tally[o] = o < n_obs ? (double)(long long)acc[o] / FIX_SCALE : 0.0;
    if (st) {
        std::memset(st, 0, sizeof(*st));
        st->packets = (int64_t)acc[ACC_PACKETS];
        st->steps = (int64_t)acc[ACC_STEPS];
        for (int q = 0; q < 8; ++q) st->ledger[q] = (double)(long long)acc[ACC_LEDGER + q] / FIX_SCALE;
        st->l_tot = info[0];
        st->n_emit_cells = (int64_t)info[1];
        st->cdf_total = info[2];
        st->flags = (int64_t)acc[ACC_FLAGS];
    }
}

// enqueue readback of accumulators and emission info into host staging buffers
gcmc_status enqueue_readback(gcmc_ctx *ctx, Plan &P, char *base, unsigned long long *h_acc, double *h_info,
                             double *info_dev)
{
    const int n = (int)P.jobs.size();
    count_launch(1);
    k_gather_info<<<(n + 127) / 128, 128, 0, ctx->stream>>>(reinterpret_cast<DevJob *>(base + P.off_jobs), n, info_dev);
    CK(cudaGetLastError());
    CK(cudaMemcpyAsync(h_acc, base + P.off_acc, (size_t)n * ACC_SLOTS * 8, cudaMemcpyDeviceToHost, ctx->stream));
    CK(cudaMemcpyAsync(h_info, info_dev, (size_t)n * 4 * sizeof(double), cudaMemcpyDeviceToHost, ctx->stream));
    return GCMC_OK;
}

__global__ void k_acc_to_tallies(const unsigned long long *acc, int n, double *out)
{
    const int q = blockIdx.x * blockDim.x + threadIdx.x;
    if (q >= n * MAX_OBS) return;
    const int j = q / MAX_OBS, o = q % MAX_OBS;
    out[q] = (double)(long long)acc[(size_t)j * ACC_SLOTS + o] / FIX_SCALE;
}

gcmc_status finish_run(gcmc_ctx *ctx, Plan &P, char *base, double *tallies_out, int tallies_memory, gcmc_stats *stats,
                       int stats_stride_jobs)
{
    const int n = (int)P.jobs.size();
    if (tallies_memory == GCMC_MEM_DEVICE && tallies_out) {
        count_launch(1);
        k_acc_to_tallies<<<(n * MAX_OBS + 127) / 128, 128, 0, ctx->stream>>>(
            reinterpret_cast<unsigned long long *>(base + P.off_acc), n, tallies_out);
        CK(cudaGetLastError());
        if (!stats) return GCMC_OK;
    }
    gcmc_status s = ensure_host(ctx, n);
    if (s) return s;
    s = enqueue_readback(ctx, P, base, ctx->h_acc, ctx->h_info, reinterpret_cast<double *>(base + P.off_gather));
    if (s) return s;
    CK(cudaStreamSynchronize(ctx->stream));
    for (int q = 0; q < n; ++q) {
        double t[MAX_OBS];
        unpack(ctx->h_acc + (size_t)q * ACC_SLOTS, ctx->h_info + 4 * q, P.jobs[q].n_tal, t,
               stats ? stats + (stats_stride_jobs ? q : 0) : nullptr);
        if (tallies_out && tallies_memory == GCMC_MEM_HOST) {
            if (stats_stride_jobs) std::memcpy(tallies_out + (size_t)q * MAX_OBS, t, sizeof(t));
            else std::memcpy(tallies_out, t, sizeof(double) * P.jobs[q].n_tal);
        }
    }
    return GCMC_OK;
}

}  // namespace

// ==================================================================== C ABI
extern "C" {

const char *gcmc_version(void) { return "gcmc 0.1 (sm_103a)"; }

gcmc_status gcmc_create(int device, gcmc_ctx **out)
{
    if (!out) return GCMC_ERR_ARG;
    *out = nullptr;
    int n = 0;
    if (cudaGetDeviceCount(&n) != cudaSuccess || device < 0 || device >= n) return GCMC_ERR_CUDA;
    if (cudaSetDevice(device) != cudaSuccess) return GCMC_ERR_CUDA;
    gcmc_ctx *ctx = new gcmc_ctx();
    ctx->device = device;
    if (cudaMalloc(&ctx->d_grids, sizeof(DevGrid) * ctx->grid_cap) != cudaSuccess) {
        delete ctx;
        return GCMC_ERR_OOM;
    }
    *out = ctx;
    return GCMC_OK;
}

gcmc_status gcmc_destroy(gcmc_ctx *ctx)
{
    if (!ctx) return GCMC_ERR_ARG;
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (auto &kv : ctx->tickets) {
        cudaEventDestroy(kv.second.done);
        cudaFreeHost(kv.second.h_acc);
        cudaFreeHost(kv.second.h_info);
        dfree(ctx, kv.second.ws);
    }
    for (auto &g : ctx->grids)
        for (void *p : g.owned) dfree(ctx, p);
    for (auto &o : ctx->opacs)
        for (void *p : o.owned) dfree(ctx, p);
    dfree(ctx, ctx->arena);
    for (auto &b : ctx->stg) {
        if (b.ptr) cudaFreeHost(b.ptr);
        if (b.ev) cudaEventDestroy(b.ev);
    }
    if (ctx->h_acc) cudaFreeHost(ctx->h_acc);
    if (ctx->h_info) cudaFreeHost(ctx->h_info);
    cudaFree(ctx->d_grids);
    delete ctx;
    return GCMC_OK;
}

gcmc_status gcmc_set_stream(gcmc_ctx *ctx, void *stream)
{
    if (!ctx) return GCMC_ERR_ARG;
    ctx->stream = (cudaStream_t)stream;
    return GCMC_OK;
}

gcmc_status gcmc_set_allocator(gcmc_ctx *ctx, gcmc_alloc_fn alloc, gcmc_free_fn free_fn, void *user)
{
    if (!ctx) return GCMC_ERR_ARG;
    if (!ctx->grids.empty() || !ctx->opacs.empty() || ctx->arena)
        return fail(ctx, GCMC_ERR_ARG, "set the allocator before the first upload");
    if ((alloc == nullptr) != (free_fn == nullptr)) return fail(ctx, GCMC_ERR_ARG, "alloc and free go together");
    ctx->alloc = alloc;
    ctx->free_fn = free_fn;
    ctx->user = user;
    return GCMC_OK;
}

const char *gcmc_last_error(gcmc_ctx *ctx) { return ctx ? ctx->err.c_str() : "no context"; }

gcmc_status gcmc_upload_grid(gcmc_ctx *ctx, const gcmc_grid_desc *d, int *grid_id)
{
    if (!ctx || !d || !grid_id) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    if (d->nlon < 1 || d->nlat < 1 || d->nr < 1) return fail(ctx, GCMC_ERR_ARG, "grid sizes must be >= 1");
    if ((int)ctx->grids.size() >= ctx->grid_cap) return fail(ctx, GCMC_ERR_RANGE, "too many grids in one context");
    const int64_t ncell = (int64_t)d->nlon * d->nlat * d->nr;
    if (ncell > ((int64_t)1 << 31) - 1) return fail(ctx, GCMC_ERR_RANGE, "more than 2^31 - 1 cells");
    // cell indices are divided by nlon and nlon * nlat with 40-bit multipliers: exact while
    // ncell * nlon * nlat < 2^40; the march tables (nr + nlat + nlon + 3 pairs) live in shared memory
    if ((double)ncell * (double)d->nlon * (double)d->nlat >= 1099511627776.0 ||
        tab_entries(d->nlon, d->nlat, d->nr) > 4096)
        return fail(ctx, GCMC_ERR_RANGE, "grid too large for this build (ncell * nlon * nlat < 2^40, nr + nlat + nlon < 4093)");
    if (!d->T || !d->p || !d->rho) return fail(ctx, GCMC_ERR_ARG, "T, p and rho are required");
    GridH G;
    if (!fetch(ctx, d->r_edges, d->nr + 1, d->memory, G.r) || !fetch(ctx, d->lat_edges, d->nlat + 1, d->memory, G.lat) ||
        !fetch(ctx, d->lon_edges, d->nlon + 1, d->memory, G.lon))
        return fail(ctx, GCMC_ERR_ARG, "edge arrays missing or unreadable");
    if (!strictly_increasing(G.r) || !(G.r[0] > 0.0)) return fail(ctx, GCMC_ERR_ARG, "r_edges must be positive, increasing");
    if (!strictly_increasing(G.lat) || G.lat.front() < -0.5 * PI - 1e-12 || G.lat.back() > 0.5 * PI + 1e-12)
        return fail(ctx, GCMC_ERR_ARG, "lat_edges must increase within [-pi/2, pi/2]");
    if (!strictly_increasing(G.lon) || std::fabs(G.lon.back() - G.lon.front() - 2.0 * PI) > 1e-9)
        return fail(ctx, GCMC_ERR_ARG, "lon_edges must increase and span 2 pi");
    // per-cell fields: validate on the host copy
    std::vector<float> T, p, rho;
    if (!fetch(ctx, d->T, ncell, d->memory, T) || !fetch(ctx, d->p, ncell, d->memory, p) ||
        !fetch(ctx, d->rho, ncell, d->memory, rho))
        return fail(ctx, GCMC_ERR_CUDA, "reading the cell fields failed");
    for (int64_t i = 0; i < ncell; ++i)
        if (!(T[i] > 0.0f) || !std::isfinite(T[i]) || !(p[i] > 0.0f) || !std::isfinite(p[i]) || !(rho[i] >= 0.0f) ||
            !std::isfinite(rho[i]))
            return fail(ctx, GCMC_ERR_NAN, "T, p must be positive and finite, rho non-negative and finite");
    const int nr = d->nr, nlat = d->nlat, nlon = d->nlon;
    std::vector<double> r2(nr + 1), slat(nlat + 1), s2lat(nlat + 1), clon(nlon + 1), slon(nlon + 1);
    std::vector<float> r_f(nr + 1), r2hi(nr + 1), r2lo(nr + 1), lat_f(nlat + 1), slat_f(nlat + 1), s2lat_f(nlat + 1),
        lon_f(nlon + 1), clon_f(nlon + 1), slon_f(nlon + 1);
    std::vector<float> shA(nr), r_lo(nr + 1), slat_lo(nlat + 1), lon_lo(nlon + 1), dslat(nlat), dlon(nlon);
    for (int k = 0; k < nr; ++k) {
        const double q = G.r[k + 1] / G.r[k];
        shA[k] = (float)(q * q * q - 1.0);
    }
    for (int k = 0; k <= nr; ++k) {
        r2[k] = G.r[k] * G.r[k];
        r_f[k] = (float)G.r[k];
        r2hi[k] = (float)r2[k];
        r2lo[k] = (float)(r2[k] - (double)r2hi[k]);
    }
    for (int j = 0; j <= nlat; ++j) {
        slat[j] = std::sin(G.lat[j]);
        s2lat[j] = slat[j] * slat[j];
        lat_f[j] = (float)G.lat[j];
        slat_f[j] = (float)slat[j];
        s2lat_f[j] = (float)s2lat[j];
    }
    for (int i = 0; i <= nlon; ++i) {
        clon[i] = std::cos(G.lon[i]);
        slon[i] = std::sin(G.lon[i]);
        lon_f[i] = (float)G.lon[i];
        clon_f[i] = (float)clon[i];
        slon_f[i] = (float)slon[i];
    }
    for (int k = 0; k <= nr; ++k) r_lo[k] = (float)(G.r[k] - (double)r_f[k]);
    for (int j = 0; j <= nlat; ++j) slat_lo[j] = (float)(slat[j] - (double)slat_f[j]);
    for (int i = 0; i <= nlon; ++i) lon_lo[i] = (float)(G.lon[i] - (double)lon_f[i]);
    for (int j = 0; j < nlat; ++j) dslat[j] = (float)(slat[j + 1] - slat[j]);
    std::vector<float> cb(nlat), cb_lo(nlat);
    for (int j = 0; j < nlat; ++j) {
        // 1 - |sin| at the band's lower edge (where the launch uniform is 0)
        const double c = slat[j] >= 0.0 ? 1.0 - slat[j] : slat[j + 1] <= 0.0 ? 1.0 + slat[j] : 0.0;
        cb[j] = (float)c;
        cb_lo[j] = (float)(c - (double)cb[j]);
    }
    for (int i = 0; i < nlon; ++i) dlon[i] = (float)(G.lon[i + 1] - G.lon[i]);
    std::vector<float2> r2p_f(nr + 1), slp_f(nlat + 1), csp_f(nlon + 1);
    std::vector<double2> r2p(nr + 1), slp(nlat + 1), csp(nlon + 1);
    for (int k = 0; k <= nr; ++k) {
        r2p_f[k] = make_float2(r2hi[k], r2lo[k]);
        r2p[k] = make_double2(r2[k], 0.0);
    }
    for (int j = 0; j <= nlat; ++j) {
        slp_f[j] = make_float2(slat_f[j], s2lat_f[j]);
        slp[j] = make_double2(slat[j], s2lat[j]);
    }
    for (int i = 0; i <= nlon; ++i) {
        csp_f[i] = make_float2(clon_f[i], slon_f[i]);
        csp[i] = make_double2(clon[i], slon[i]);
    }
    std::vector<double> vol(ncell);
    for (int64_t idx = 0; idx < ncell; ++idx) {
        const int64_t i = idx % nlon, j = (idx / nlon) % nlat, k = idx / ((int64_t)nlon * nlat);
        const double r1 = G.r[k], r2v = G.r[k + 1];
        vol[idx] = (r2v * r2v * r2v - r1 * r1 * r1) / 3.0 * (std::sin(G.lat[j + 1]) - std::sin(G.lat[j])) *
                   (G.lon[i + 1] - G.lon[i]);
    }
    cudaSetDevice(ctx->device);
    cudaError_t e = cudaSuccess;
    DevGrid &g = G.dg;
    g.nlon = nlon;
    g.nlat = nlat;
    g.nr = nr;
    g.ncell = ncell;
    g.R0 = G.r[0];
    g.Rtoa = G.r[nr];
    g.lon0 = G.lon[0];
    g.r = dput(ctx, G.owned, G.r.data(), nr + 1, e);
    g.r2 = dput(ctx, G.owned, r2.data(), nr + 1, e);
    g.lat = dput(ctx, G.owned, G.lat.data(), nlat + 1, e);
    g.slat = dput(ctx, G.owned, slat.data(), nlat + 1, e);
    g.s2lat = dput(ctx, G.owned, s2lat.data(), nlat + 1, e);
    g.lon = dput(ctx, G.owned, G.lon.data(), nlon + 1, e);
    g.clon = dput(ctx, G.owned, clon.data(), nlon + 1, e);
    g.slon = dput(ctx, G.owned, slon.data(), nlon + 1, e);
    g.r_f = dput(ctx, G.owned, r_f.data(), nr + 1, e);
    g.r2hi_f = dput(ctx, G.owned, r2hi.data(), nr + 1, e);
    g.r2lo_f = dput(ctx, G.owned, r2lo.data(), nr + 1, e);
    g.lat_f = dput(ctx, G.owned, lat_f.data(), nlat + 1, e);
    g.slat_f = dput(ctx, G.owned, slat_f.data(), nlat + 1, e);
    g.s2lat_f = dput(ctx, G.owned, s2lat_f.data(), nlat + 1, e);
    g.lon_f = dput(ctx, G.owned, lon_f.data(), nlon + 1, e);
    g.clon_f = dput(ctx, G.owned, clon_f.data(), nlon + 1, e);
    g.slon_f = dput(ctx, G.owned, slon_f.data(), nlon + 1, e);
    g.shA_f = dput(ctx, G.owned, shA.data(), nr, e);
    g.r_lo_f = dput(ctx, G.owned, r_lo.data(), nr + 1, e);
    g.slat_lo_f = dput(ctx, G.owned, slat_lo.data(), nlat + 1, e);
    g.lon_lo_f = dput(ctx, G.owned, lon_lo.data(), nlon + 1, e);
    g.dslat_f = dput(ctx, G.owned, dslat.data(), nlat, e);
    g.cb_f = dput(ctx, G.owned, cb.data(), nlat, e);
    g.cb_lo_f = dput(ctx, G.owned, cb_lo.data(), nlat, e);
    g.dlon_f = dput(ctx, G.owned, dlon.data(), nlon, e);
    g.r2p_f = dput(ctx, G.owned, r2p_f.data(), nr + 1, e);
    g.slp_f = dput(ctx, G.owned, slp_f.data(), nlat + 1, e);
    g.csp_f = dput(ctx, G.owned, csp_f.data(), nlon + 1, e);
    g.r2p = dput(ctx, G.owned, r2p.data(), nr + 1, e);
    g.slp = dput(ctx, G.owned, slp.data(), nlat + 1, e);
    g.csp = dput(ctx, G.owned, csp.data(), nlon + 1, e);
    g.mag_lon = (((uint64_t)1 << 40) + (uint64_t)nlon - 1) / (uint64_t)nlon;
    g.mag_ll = (((uint64_t)1 << 40) + (uint64_t)nlon * nlat - 1) / ((uint64_t)nlon * nlat);
    g.T = dput(ctx, G.owned, d->T, ncell, e);
    g.p = dput(ctx, G.owned, d->p, ncell, e);
    g.rho = dput(ctx, G.owned, d->rho, ncell, e);
    g.wind = d->wind ? dput(ctx, G.owned, d->wind, 3 * ncell, e) : nullptr;
    g.vol = dput(ctx, G.owned, vol.data(), ncell, e);
    if (e != cudaSuccess) {
        for (void *q : G.owned) dfree(ctx, q);
        return e == cudaErrorMemoryAllocation ? fail(ctx, GCMC_ERR_OOM, "grid allocation failed")
                                              : cuda_fail(ctx, e, "grid upload");
    }
    const int id = (int)ctx->grids.size();
    CK(cudaMemcpyAsync(ctx->d_grids + id, &G.dg, sizeof(DevGrid), cudaMemcpyHostToDevice, ctx->stream));
    CK(cudaStreamSynchronize(ctx->stream));   // host staging vectors go out of scope
    ctx->grids.push_back(std::move(G));
    *grid_id = id;
    return GCMC_OK;
}

gcmc_status gcmc_upload_opacity(gcmc_ctx *ctx, int grid_id, const gcmc_opacity_desc *d, int *opac_id)
{
    if (!ctx || !d || !opac_id) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    if (grid_id < 0 || grid_id >= (int)ctx->grids.size()) return fail(ctx, GCMC_ERR_ARG, "bad grid_id");
    cudaSetDevice(ctx->device);
    const int64_t ncell = ctx->grids[grid_id].dg.ncell;
    OpacH O;
    O.kind = d->kind;
    O.grid = grid_id;
    cudaError_t e = cudaSuccess;
    auto finite_nonneg = [](const std::vector<double> &v) {
        for (double x : v)
            if (!(x >= 0.0) || !std::isfinite(x)) return false;
        return true;
    };
    if (d->kind == GCMC_OPAC_ALBEDO) {
        if (d->nlam < 1) return fail(ctx, GCMC_ERR_ARG, "nlam must be >= 1");
        std::vector<double> ka, kr, qc, wc, gc;
        if (!fetch(ctx, d->kabs, d->nlam, d->memory, ka) || !fetch(ctx, d->kray, d->nlam, d->memory, kr) ||
            !fetch(ctx, d->qcld, d->nlam, d->memory, qc) || !fetch(ctx, d->wcld, d->nlam, d->memory, wc) ||
            !fetch(ctx, d->gcld, d->nlam, d->memory, gc))
            return fail(ctx, GCMC_ERR_ARG, "albedo opacity arrays missing");
        if (!finite_nonneg(ka) || !finite_nonneg(kr) || !finite_nonneg(qc) || !finite_nonneg(wc))
            return fail(ctx, GCMC_ERR_NAN, "negative or non-finite opacity");
        for (int l = 0; l < d->nlam; ++l)
            if (!(wc[l] <= 1.0) || !(gc[l] > -1.0 && gc[l] < 1.0)) return fail(ctx, GCMC_ERR_ARG, "wcld in [0,1], |gcld| < 1");
        if (d->acld) {
            std::vector<float> ac;
            if (!fetch(ctx, d->acld, ncell, d->memory, ac)) return fail(ctx, GCMC_ERR_CUDA, "reading acld failed");
            for (float x : ac)
                if (!(x >= 0.0f) || !std::isfinite(x)) return fail(ctx, GCMC_ERR_NAN, "negative or non-finite acld");
        }
        O.nlam = d->nlam;
        O.alb.nlam = d->nlam;
        O.alb.kabs = dput(ctx, O.owned, ka.data(), d->nlam, e);
        O.alb.kray = dput(ctx, O.owned, kr.data(), d->nlam, e);
        O.alb.qcld = dput(ctx, O.owned, qc.data(), d->nlam, e);
        O.alb.wcld = dput(ctx, O.owned, wc.data(), d->nlam, e);
        O.alb.gcld = dput(ctx, O.owned, gc.data(), d->nlam, e);
        O.alb.acld = d->acld ? dput(ctx, O.owned, d->acld, ncell, e) : nullptr;
    } else if (d->kind == GCMC_OPAC_KTABLE || d->kind == GCMC_OPAC_XSEC) {
        if (d->nT < 2 || d->np < 2) return fail(ctx, GCMC_ERR_ARG, "table axes need >= 2 points");
        std::vector<double> Tg, pg;
        if (!fetch(ctx, d->Tg, d->nT, d->memory, Tg) || !fetch(ctx, d->pg, d->np, d->memory, pg))
            return fail(ctx, GCMC_ERR_ARG, "table axes missing");
        if (!strictly_increasing(Tg) || !strictly_increasing(pg) || !(Tg[0] > 0) || !(pg[0] > 0))
            return fail(ctx, GCMC_ERR_ARG, "table axes must be positive and increasing");
        if (d->kind == GCMC_OPAC_KTABLE) {
            if (d->nb < 1 || d->ng < 1) return fail(ctx, GCMC_ERR_ARG, "nb, ng must be >= 1");
            const size_t nk = (size_t)d->nb * d->ng * d->nT * d->np;
            std::vector<float> k;
            std::vector<double> lam;
            if (!fetch(ctx, d->k, nk, d->memory, k) || !fetch(ctx, d->lam, d->nb, d->memory, lam))
                return fail(ctx, GCMC_ERR_ARG, "k-table arrays missing");
            std::vector<double> lnk(nk);
            for (size_t i = 0; i < nk; ++i) {
                if (!(k[i] > 0.0f) || !std::isfinite(k[i])) return fail(ctx, GCMC_ERR_NAN, "k must be positive, finite");
                lnk[i] = std::log((double)k[i]);
            }
            for (double l : lam)
                if (!(l > 0.0)) return fail(ctx, GCMC_ERR_ARG, "band wavelengths must be positive");
            O.kt.nb = d->nb;
            O.kt.ng = d->ng;
            O.kt.nT = d->nT;
            O.kt.np = d->np;
            // FP32 node records for FP32 marches: {k_ab, d1, d2, d3} with the differences of ln k taken in FP64
            std::vector<float4> node(nk);
            const int nT = d->nT, np = d->np;
            for (size_t sl = 0; sl < (size_t)d->nb * d->ng; ++sl)
                for (int a = 0; a < nT; ++a)
                    for (int b = 0; b < np; ++b) {
                        const size_t i = sl * nT * np + (size_t)a * np + b;
                        const int a1 = a + 1 < nT ? a + 1 : a, b1 = b + 1 < np ? b + 1 : b;
                        const double l00 = lnk[i], l10 = lnk[sl * nT * np + (size_t)a1 * np + b];
                        const double l01 = lnk[sl * nT * np + (size_t)a * np + b1];
                        const double l11 = lnk[sl * nT * np + (size_t)a1 * np + b1];
                        node[i] = make_float4(k[i], (float)(l10 - l00), (float)(l01 - l00), (float)(l11 - l10 - l01 + l00));
                    }
            O.kt.gw = nullptr;
            if (d->gw) {
                std::vector<double> gw;
                if (!fetch(ctx, d->gw, d->ng, d->memory, gw)) return fail(ctx, GCMC_ERR_ARG, "g weights missing");
                double sw = 0.0;
                for (double w : gw) {
                    if (!(w >= 0.0) || !std::isfinite(w)) return fail(ctx, GCMC_ERR_ARG, "g weights must be >= 0");
                    sw += w;
                }
                if (!(sw > 0.0)) return fail(ctx, GCMC_ERR_ARG, "g weights sum to 0");
                O.kt.gw = dput(ctx, O.owned, gw.data(), d->ng, e);
            }
            O.kt.lnk = dput(ctx, O.owned, lnk.data(), nk, e);
            O.kt.node_f = dput(ctx, O.owned, node.data(), nk, e);
            O.kt.Tg = dput(ctx, O.owned, Tg.data(), d->nT, e);
            O.kt.pg = dput(ctx, O.owned, pg.data(), d->np, e);
            O.lam = lam;
            O.nlam = d->nb;
            // per-cell tables on this grid: interpolation cells and weights, 4 pi V B(T) per band
            const DevGrid &hg = ctx->grids[grid_id].dg;
            const double *lam_dev = dput(ctx, O.owned, lam.data(), d->nb, e);
            int2 *ab = dput<int2>(ctx, O.owned, nullptr, hg.ncell, e);
            double2 *w64 = dput<double2>(ctx, O.owned, nullptr, hg.ncell, e);
            float2 *w32 = dput<float2>(ctx, O.owned, nullptr, hg.ncell, e);
            double *vb = dput<double>(ctx, O.owned, nullptr, (size_t)d->nb * hg.ncell, e);
            if (e == cudaSuccess) e = ktable_cells(hg, lam_dev, d->nb, ab, w64, w32, vb, O.kt, ctx->stream);
            O.kt.ab = ab;
            O.kt.w64 = w64;
            O.kt.w32 = w32;
            O.kt.vb = vb;
        } else {
            if (d->nl < 2) return fail(ctx, GCMC_ERR_ARG, "xsec table needs >= 2 wavelengths");
            const size_t ns = (size_t)d->nl * d->nT * d->np;
            std::vector<float> sg;
            std::vector<double> xl;
            if (!fetch(ctx, d->sigma, ns, d->memory, sg) || !fetch(ctx, d->xlam, d->nl, d->memory, xl))
                return fail(ctx, GCMC_ERR_ARG, "xsec arrays missing");
            if (!strictly_increasing(xl) || !(xl[0] > 0)) return fail(ctx, GCMC_ERR_ARG, "xlam must increase");
            std::vector<double> ls(ns);
            std::vector<float> lsf(ns);
            for (size_t i = 0; i < ns; ++i) {
                if (!(sg[i] > 0.0f) || !std::isfinite(sg[i])) return fail(ctx, GCMC_ERR_NAN, "sigma must be positive");
                ls[i] = std::log((double)sg[i]);
                lsf[i] = (float)ls[i];
            }
            O.xs.nl = d->nl;
            O.xs.nT = d->nT;
            O.xs.np = d->np;
            O.xs.lam = dput(ctx, O.owned, xl.data(), d->nl, e);
            O.xs.lnsig = dput(ctx, O.owned, ls.data(), ns, e);
            O.xs.lnsig_f = dput(ctx, O.owned, lsf.data(), ns, e);
            O.xs.Tg = dput(ctx, O.owned, Tg.data(), d->nT, e);
            O.xs.pg = dput(ctx, O.owned, pg.data(), d->np, e);
            O.xs.view_theta = d->view_theta;
            O.xs.view_phi = d->view_phi;
            O.xs.omega_rot = d->omega_rot;
            O.lam = xl;
            O.nlam = d->nl;
            // per-cell tables on this grid: interpolation cells and weights, Doppler factors
            const DevGrid &hg = ctx->grids[grid_id].dg;
            int2 *ab = dput<int2>(ctx, O.owned, nullptr, hg.ncell, e);
            double2 *w = dput<double2>(ctx, O.owned, nullptr, hg.ncell, e);
            double *fac = dput<double>(ctx, O.owned, nullptr, hg.ncell, e);
            float2 *w32 = dput<float2>(ctx, O.owned, nullptr, hg.ncell, e);
            float *dlt = dput<float>(ctx, O.owned, nullptr, hg.ncell, e);
            float *mm = dput<float>(ctx, O.owned, nullptr, 2, e);
            if (e == cudaSuccess) e = xsec_cells(hg, O.xs, ab, w, fac, w32, dlt, mm, ctx->stream);
            float hmm[2] = {0.0f, 0.0f};
            if (e == cudaSuccess) e = cudaMemcpyAsync(hmm, mm, sizeof(hmm), cudaMemcpyDeviceToHost, ctx->stream);
            if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
            O.xs.ab = ab;
            O.xs.w = w;
            O.xs.fac = fac;
            O.xs.w32 = w32;
            O.xs.dlt_f = dlt;
            O.xs.dmin = hmm[0];
            O.xs.dmax = hmm[1];
        }
    } else {
        return fail(ctx, GCMC_ERR_ARG, "unknown opacity kind");
    }
    if (e != cudaSuccess) {
        for (void *q : O.owned) dfree(ctx, q);
        return e == cudaErrorMemoryAllocation ? fail(ctx, GCMC_ERR_OOM, "opacity allocation failed")
                                              : cuda_fail(ctx, e, "opacity upload");
    }
    CK(cudaStreamSynchronize(ctx->stream));
    *opac_id = (int)ctx->opacs.size();
    ctx->opacs.push_back(std::move(O));
    return GCMC_OK;
}

gcmc_status gcmc_set_source(gcmc_ctx *ctx, int grid_id, const gcmc_source_desc *d, int *source_id)
{
    if (!ctx || !d || !source_id) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    if (grid_id < 0 || grid_id >= (int)ctx->grids.size()) return fail(ctx, GCMC_ERR_ARG, "bad grid_id");
    if (d->n_obs < 1 || d->n_obs > GCMC_MAX_OBS) return fail(ctx, GCMC_ERR_ARG, "n_obs must be in 1..GCMC_MAX_OBS");
    auto unit = [](const double *v) { return std::fabs(v[0] * v[0] + v[1] * v[1] + v[2] * v[2] - 1.0) < 1e-9; };
    if (!unit(d->star)) return fail(ctx, GCMC_ERR_ARG, "star must be a unit vector");
    for (int o = 0; o < d->n_obs; ++o)
        if (!unit(d->obs[o])) return fail(ctx, GCMC_ERR_ARG, "observer directions must be unit vectors");
    if (!(d->p_surv > 0.0 && d->p_surv <= 1.0) || !(d->w_rr >= 0.0) || !(d->tau_peel_cut > 0.0) ||
        !(d->beta_emis >= 0.0 && d->beta_emis <= 1.0) || !(d->tau_vert_max > 0.0))
        return fail(ctx, GCMC_ERR_ARG, "options out of range");
    if (d->cloud_phase != GCMC_CLOUD_HG && d->cloud_phase != GCMC_CLOUD_TTHG)
        return fail(ctx, GCMC_ERR_ARG, "unknown cloud_phase");
    if (!(d->surface_albedo >= 0.0 && d->surface_albedo <= 1.0))
        return fail(ctx, GCMC_ERR_ARG, "surface_albedo must be in [0, 1]");
    if (d->ld_law < GCMC_LD_NONE || d->ld_law > GCMC_LD_CLARET4) return fail(ctx, GCMC_ERR_ARG, "unknown ld_law");
    if (d->ld_law != GCMC_LD_NONE && !(d->star_radius > 0.0))
        return fail(ctx, GCMC_ERR_ARG, "limb darkening needs star_radius > 0");
    if (!(d->star_dist == 0.0 || d->star_dist > d->star_radius))
        return fail(ctx, GCMC_ERR_ARG, "star_dist must be 0 or above star_radius");
    for (int c = 0; c < 4; ++c)
        if (!std::isfinite(d->ld_coef[c])) return fail(ctx, GCMC_ERR_ARG, "limb-darkening coefficients must be finite");
    if (d->g_bias < GCMC_GBIAS_NONE || d->g_bias > GCMC_GBIAS_COMPOSITE) return fail(ctx, GCMC_ERR_ARG, "unknown g_bias");
    if (d->forced_first < 0 || d->forced_first > 2 || (d->cont_abs != 0 && d->cont_abs != 1) || d->path_bias < 0 ||
        d->path_bias > 2)
        return fail(ctx, GCMC_ERR_ARG, "forced_first and path_bias are 0, 1 or 2; cont_abs 0 or 1");
    if (!(d->g_beta >= 0.0 && d->g_beta <= 1.0)) return fail(ctx, GCMC_ERR_ARG, "g_beta must be in [0, 1]");
    *source_id = (int)ctx->sources.size();
    ctx->sources.push_back(*d);
    return GCMC_OK;
}

gcmc_status gcmc_run_packets(gcmc_ctx *ctx, const gcmc_job *job, double *tallies_out, int tallies_memory,
                             gcmc_stats *stats_out)
{
    if (!ctx || !job) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    cudaSetDevice(ctx->device);
    Plan P;
    gcmc_status s = plan_run(ctx, job, 1, 128, P);
    if (s) return s;
    if ((s = ensure_arena(ctx, P.ws_bytes))) return s;
    char *base = (char *)ctx->arena;
    prof_mark(ctx);
    if ((s = stage(ctx, P, base))) return s;
    prof_mark(ctx);
    const DevJob *dj = reinterpret_cast<const DevJob *>(base + P.off_jobs);
    cudaError_t e = launch_plain(P.jobs[0].precision, P.scatter, P.feat, ctx->d_grids, dj, 0, job->n_packets, nullptr, P.tab_n,
                                 ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "transport launch");
    prof_mark(ctx);
    return finish_run(ctx, P, base, tallies_out, tallies_memory, stats_out, 0);
}

gcmc_status gcmc_run_batch(gcmc_ctx *ctx, const gcmc_job *jobs, int n_jobs, const gcmc_launch_cfg *cfg,
                           double *tallies_out, int tallies_memory, gcmc_stats *stats_out)
{
    if (!ctx || !jobs) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    cudaSetDevice(ctx->device);
    const int chunk = cfg && cfg->chunk > 0 ? cfg->chunk : 1024;
    Plan P;
    gcmc_status s = plan_run(ctx, jobs, n_jobs, chunk, P);
    if (s) return s;
    if ((s = ensure_arena(ctx, P.ws_bytes))) return s;
    char *base = (char *)ctx->arena;
    int prec = P.jobs[0].precision;
    for (const DevJob &d : P.jobs)
        if (d.precision != prec) return fail(ctx, GCMC_ERR_ARG, "a batch runs in one precision");
    prof_mark(ctx);
    if ((s = stage(ctx, P, base))) return s;
    prof_mark(ctx);
    const DevJob *dj = reinterpret_cast<const DevJob *>(base + P.off_jobs);
    cudaError_t e = launch_persistent(prec, P.scatter, P.feat, ctx->d_grids, dj, n_jobs, P.total_items, chunk, cfg ? cfg->block : 0,
                                      cfg ? cfg->blocks_per_sm : 0, cfg && cfg->interval > 0 ? cfg->interval : 1,
                                      cfg && cfg->refill_min > 0 ? cfg->refill_min : 16, P.one_grid, P.tab_n,
                                      reinterpret_cast<unsigned long long *>(base + P.off_work), ctx->stream);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "transport launch");
    prof_mark(ctx);
    return finish_run(ctx, P, base, tallies_out, tallies_memory, stats_out, 1);
}

gcmc_status gcmc_run_contrib(gcmc_ctx *ctx, const gcmc_job *job, double *tallies_out, double *cf_out,
                             gcmc_stats *stats_out)
{
    if (!ctx || !job || !cf_out) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    if (job->mode == GCMC_TRANSMISSION)
        return fail(ctx, GCMC_ERR_ARG, "contribution functions are defined for albedo and emission jobs");
    cudaSetDevice(ctx->device);
    const int chunk = 256;
    Plan P;
    gcmc_status s = plan_run(ctx, job, 1, chunk, P);
    if (s) return s;
    if ((s = ensure_arena(ctx, P.ws_bytes))) return s;
    char *base = (char *)ctx->arena;
    const int64_t ncell = ctx->grids[job->grid_id].dg.ncell;
    const size_t ncf = (size_t)2 * P.jobs[0].n_obs * ncell;
    unsigned long long *dcf = (unsigned long long *)dalloc(ctx, ncf * 8);
    if (!dcf) return fail(ctx, GCMC_ERR_OOM, "contribution-function counters");
    cudaError_t e = cudaMemsetAsync(dcf, 0, ncf * 8, ctx->stream);
    P.jobs[0].cf = dcf;
    P.jobs[0].cf_ncell = ncell;
    if (e == cudaSuccess && (s = stage(ctx, P, base)) == GCMC_OK) {
        const DevJob *dj = reinterpret_cast<const DevJob *>(base + P.off_jobs);
        e = launch_persistent(P.jobs[0].precision, P.scatter, P.feat, ctx->d_grids, dj, 1, P.total_items, chunk, 128, 0, 4, 8,
                              P.one_grid, P.tab_n, reinterpret_cast<unsigned long long *>(base + P.off_work), ctx->stream);
    }
    std::vector<unsigned long long> h(ncf);
    if (!s && e == cudaSuccess) e = cudaMemcpyAsync(h.data(), dcf, ncf * 8, cudaMemcpyDeviceToHost, ctx->stream);
    if (!s && e == cudaSuccess) s = finish_run(ctx, P, base, tallies_out, GCMC_MEM_HOST, stats_out, 0);
    if (e != cudaSuccess && !s) s = cuda_fail(ctx, e, "contribution-function run");
    cudaStreamSynchronize(ctx->stream);
    dfree(ctx, dcf);
    if (s) return s;
    for (size_t i = 0; i < ncf; ++i) cf_out[i] = (double)(long long)h[i] / FIX_SCALE;
    return GCMC_OK;
}

gcmc_status gcmc_submit(gcmc_ctx *ctx, const gcmc_job *jobs, int n_jobs, const gcmc_launch_cfg *cfg, uint64_t *ticket)
{
    if (!ctx || !jobs || !ticket) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    cudaSetDevice(ctx->device);
    const int chunk = cfg && cfg->chunk > 0 ? cfg->chunk : 1024;
    Plan P;
    gcmc_status s = plan_run(ctx, jobs, n_jobs, chunk, P);
    if (s) return s;
    int prec = P.jobs[0].precision;
    for (const DevJob &d : P.jobs)
        if (d.precision != prec) return fail(ctx, GCMC_ERR_ARG, "a batch runs in one precision");
    Ticket T;
    T.n_jobs = n_jobs;
    T.ws = dalloc(ctx, P.ws_bytes);
    if (!T.ws) return fail(ctx, GCMC_ERR_OOM, "ticket workspace");
    char *base = (char *)T.ws;
    if ((s = stage(ctx, P, base))) {
        dfree(ctx, T.ws);
        return s;
    }
    const DevJob *dj = reinterpret_cast<const DevJob *>(base + P.off_jobs);
    cudaError_t e = launch_persistent(prec, P.scatter, P.feat, ctx->d_grids, dj, n_jobs, P.total_items, chunk, cfg ? cfg->block : 0,
                                      cfg ? cfg->blocks_per_sm : 0, cfg && cfg->interval > 0 ? cfg->interval : 1,
                                      cfg && cfg->refill_min > 0 ? cfg->refill_min : 16, P.one_grid, P.tab_n,
                                      reinterpret_cast<unsigned long long *>(base + P.off_work), ctx->stream);
    if (e != cudaSuccess) {
        dfree(ctx, T.ws);
        return cuda_fail(ctx, e, "transport launch");
    }
    CK(cudaMallocHost((void **)&T.h_acc, (size_t)n_jobs * ACC_SLOTS * 8));
    CK(cudaMallocHost((void **)&T.h_info, (size_t)n_jobs * 4 * sizeof(double)));
    if ((s = enqueue_readback(ctx, P, base, T.h_acc, T.h_info, reinterpret_cast<double *>(base + P.off_gather)))) return s;
    CK(cudaEventCreateWithFlags(&T.done, cudaEventDisableTiming));
    CK(cudaEventRecord(T.done, ctx->stream));
    const uint64_t id = ctx->next_ticket++;
    ctx->tickets[id] = T;
    *ticket = id;
    return GCMC_OK;
}

gcmc_status gcmc_poll(gcmc_ctx *ctx, uint64_t ticket, double *tallies_out, gcmc_stats *stats_out)
{
    if (!ctx) return GCMC_ERR_ARG;
    auto it = ctx->tickets.find(ticket);
    if (it == ctx->tickets.end()) return fail(ctx, GCMC_ERR_ARG, "unknown ticket");
    Ticket &T = it->second;
    const cudaError_t q = cudaEventQuery(T.done);
    if (q == cudaErrorNotReady) return GCMC_ERR_NOT_READY;
    if (q != cudaSuccess) return cuda_fail(ctx, q, "ticket");
    for (int j = 0; j < T.n_jobs; ++j) {
        double t[MAX_OBS];
        // n_obs is not kept with the ticket: unused observer slots are zero
        unpack(T.h_acc + (size_t)j * ACC_SLOTS, T.h_info + 4 * j, MAX_OBS, t, stats_out ? stats_out + j : nullptr);
        if (tallies_out) std::memcpy(tallies_out + (size_t)j * MAX_OBS, t, sizeof(t));
    }
    cudaEventDestroy(T.done);
    cudaFreeHost(T.h_acc);
    cudaFreeHost(T.h_info);
    dfree(ctx, T.ws);
    ctx->tickets.erase(it);
    return GCMC_OK;
}

gcmc_status gcmc_job_columns(gcmc_ctx *ctx, const gcmc_job *job, int32_t *n_cols)
{
    if (!ctx || !job || !n_cols) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    const gcmc_status s = check_job(ctx, *job);
    if (s) return s;
    *n_cols = job_columns(ctx, *job);
    return GCMC_OK;
}

gcmc_status gcmc_run_packets_debug(gcmc_ctx *ctx, const gcmc_job *job, int64_t packet0, int64_t n_run, double *pk_f,
                                   int32_t pk_f_cols, int64_t *pk_steps, double *pk_tau, int32_t n_trace,
                                   int32_t max_trace, int32_t *tr_cell, double *tr_len, int32_t *tr_n, double *tallies_out,
                                   gcmc_stats *stats_out)
{
    if (!ctx || !job) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    if (packet0 < 0 || n_run < 0 || packet0 + n_run > job->n_packets) return fail(ctx, GCMC_ERR_ARG, "packet range");
    if (n_trace < 0 || max_trace < 0 || n_trace > n_run) return fail(ctx, GCMC_ERR_ARG, "trace sizes");
    cudaSetDevice(ctx->device);
    Plan P;
    gcmc_status s = plan_run(ctx, job, 1, 128, P);
    if (s) return s;
    if (pk_f && pk_f_cols < P.jobs[0].n_tal) return fail(ctx, GCMC_ERR_ARG, "pk_f has fewer columns than the job tallies");
    if ((s = ensure_arena(ctx, P.ws_bytes))) return s;
    char *base = (char *)ctx->arena;
    if ((s = stage(ctx, P, base))) return s;
    const int nobs = P.jobs[0].n_tal;
    HostLog hl{};
    std::vector<void *> tmp;
    cudaError_t e = cudaSuccess;
    auto zalloc = [&](size_t bytes) -> void * {
        void *p = dalloc(ctx, bytes);
        if (p) {
            tmp.push_back(p);
            if (cudaMemsetAsync(p, 0, bytes, ctx->stream) != cudaSuccess) e = cudaErrorUnknown;
        } else {
            e = cudaErrorMemoryAllocation;
        }
        return p;
    };
    hl.pk_f = (double *)zalloc((size_t)n_run * nobs * sizeof(double));
    hl.pk_steps = (int64_t *)zalloc((size_t)n_run * sizeof(int64_t));
    hl.pk_tau = (double *)zalloc((size_t)n_run * sizeof(double));
    hl.n_trace = n_trace;
    hl.max_trace = max_trace;
    if (n_trace > 0 && max_trace > 0) {
        hl.tr_cell = (int32_t *)zalloc((size_t)n_trace * max_trace * sizeof(int32_t));
        hl.tr_len = (double *)zalloc((size_t)n_trace * max_trace * sizeof(double));
        hl.tr_n = (int32_t *)zalloc((size_t)n_trace * sizeof(int32_t));
    }
    if (e == cudaSuccess) {
        const DevJob *dj = reinterpret_cast<const DevJob *>(base + P.off_jobs);
        e = launch_plain(P.jobs[0].precision, P.scatter, P.feat, ctx->d_grids, dj, packet0, n_run, &hl, P.tab_n, ctx->stream);
    }
    if (e == cudaSuccess) {
        if (pk_f && n_run > 0)
            e = cudaMemcpy2DAsync(pk_f, (size_t)pk_f_cols * 8, hl.pk_f, (size_t)nobs * 8, (size_t)nobs * 8, (size_t)n_run,
                                  cudaMemcpyDeviceToHost, ctx->stream);
        if (pk_steps && e == cudaSuccess)
            e = cudaMemcpyAsync(pk_steps, hl.pk_steps, (size_t)n_run * 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (pk_tau && e == cudaSuccess)
            e = cudaMemcpyAsync(pk_tau, hl.pk_tau, (size_t)n_run * 8, cudaMemcpyDeviceToHost, ctx->stream);
        if (hl.tr_cell && e == cudaSuccess) {
            if (tr_cell) e = cudaMemcpyAsync(tr_cell, hl.tr_cell, (size_t)n_trace * max_trace * 4, cudaMemcpyDeviceToHost, ctx->stream);
            if (tr_len && e == cudaSuccess)
                e = cudaMemcpyAsync(tr_len, hl.tr_len, (size_t)n_trace * max_trace * 8, cudaMemcpyDeviceToHost, ctx->stream);
            if (tr_n && e == cudaSuccess) e = cudaMemcpyAsync(tr_n, hl.tr_n, (size_t)n_trace * 4, cudaMemcpyDeviceToHost, ctx->stream);
        }
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    for (void *p : tmp) dfree(ctx, p);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "debug run");
    return finish_run(ctx, P, base, tallies_out, GCMC_MEM_HOST, stats_out, 0);
}

gcmc_status gcmc_prep_cells(gcmc_ctx *ctx, const gcmc_job *job, double *alpha, double *omega, double *g, double *pgas,
                            double *lum, double *cdf, double *wcell, gcmc_stats *stats_out)
{
    if (!ctx || !job) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    if (job->mode == GCMC_EMISSION && job->g_idx < 0)
        return fail(ctx, GCMC_ERR_ARG, "cell tables are per g-ordinate: give g_idx >= 0");
    cudaSetDevice(ctx->device);
    Plan P;
    gcmc_status s = plan_run(ctx, job, 1, 128, P);
    if (s) return s;
    if ((s = ensure_arena(ctx, P.ws_bytes))) return s;
    char *base = (char *)ctx->arena;
    const int64_t ncell = ctx->grids[job->grid_id].dg.ncell;
    double *dlum = nullptr;
    if (lum && job->mode == GCMC_EMISSION) {
        dlum = (double *)dalloc(ctx, ncell * 8);
        if (!dlum) return fail(ctx, GCMC_ERR_OOM, "lum");
    }
    if ((s = stage(ctx, P, base, dlum))) {
        dfree(ctx, dlum);
        return s;
    }
    const bool f64 = P.jobs[0].precision == GCMC_FP64;
    const size_t esz = f64 ? 8 : 4;
    const int nrec = P.jobs[0].rec4 ? 4 : 1;
    std::vector<char> raw(ncell * nrec * esz);
    CK(cudaMemcpyAsync(raw.data(), base + P.off_rec[0], raw.size(), cudaMemcpyDeviceToHost, ctx->stream));
    std::vector<long long> cq;
    std::vector<char> wraw;
    if (job->mode == GCMC_EMISSION) {
        if (cdf) {
            cq.resize(ncell);
            CK(cudaMemcpyAsync(cq.data(), base + P.off_cdf[0], ncell * 8, cudaMemcpyDeviceToHost, ctx->stream));
        }
        if (wcell) {
            wraw.resize(ncell * esz);
            CK(cudaMemcpyAsync(wraw.data(), base + P.off_w[0], wraw.size(), cudaMemcpyDeviceToHost, ctx->stream));
        }
        if (dlum) CK(cudaMemcpyAsync(lum, dlum, ncell * 8, cudaMemcpyDeviceToHost, ctx->stream));
    }
    s = finish_run(ctx, P, base, nullptr, GCMC_MEM_HOST, stats_out, 0);
    dfree(ctx, dlum);
    if (s) return s;
    // the cumulative pdf as the fraction-scaled value Q / 2^62, the weights widened to FP64
    for (size_t i = 0; i < cq.size(); ++i) cdf[i] = (double)cq[i] / 4611686018427387904.0;
    if (!wraw.empty())
        for (int64_t i = 0; i < ncell; ++i)
            wcell[i] = f64 ? reinterpret_cast<const double *>(wraw.data())[i]
                           : (double)reinterpret_cast<const float *>(wraw.data())[i];
    for (int64_t i = 0; i < ncell; ++i) {
        double v[4] = {0, 0, 0, 0};
        for (int c = 0; c < nrec; ++c)
            v[c] = f64 ? reinterpret_cast<double *>(raw.data())[i * nrec + c] : reinterpret_cast<float *>(raw.data())[i * nrec + c];
        if (alpha) alpha[i] = v[0];
        if (nrec == 4) {
            if (omega) omega[i] = v[1];
            if (g) g[i] = v[2];
            if (pgas) pgas[i] = v[3];
        }
    }
    return GCMC_OK;
}

gcmc_status gcmc_postscale(gcmc_ctx *ctx, int grid_id, int mode, double tally, int64_t n_packets, double l_tot,
                           gcmc_observables *out)
{
    if (!ctx || !out) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    if (grid_id < 0 || grid_id >= (int)ctx->grids.size()) return fail(ctx, GCMC_ERR_ARG, "bad grid_id");
    if (n_packets <= 0) return fail(ctx, GCMC_ERR_ARG, "n_packets must be positive");
    std::memset(out, 0, sizeof(*out));
    const double R0 = ctx->grids[grid_id].dg.R0, Rt = ctx->grids[grid_id].dg.Rtoa;
    const double N = (double)n_packets;
    if (mode == GCMC_ALBEDO) {
        out->S = tally / N;
        out->A_g = PI * out->S;
        out->A_g_R0 = out->A_g * (Rt / R0) * (Rt / R0);
    } else if (mode == GCMC_EMISSION) {
        out->L_p = l_tot / N * tally;
        out->I_p = out->L_p / (PI * Rt * Rt);
        out->F_p = PI * out->I_p;
    } else if (mode == GCMC_TRANSMISSION) {
        out->I_p = (Rt - R0) / N * Rt * tally;
        out->area = R0 * R0 + 2.0 * out->I_p;
    } else {
        return fail(ctx, GCMC_ERR_ARG, "bad mode");
    }
    return GCMC_OK;
}

// stellar limb darkening I(mu)/I(disk centre) of the laws of gcmc_source_desc, before clipping at 0
static double limb_raw(int law, const double *c, double mu)
{
    const double x = 1.0 - mu;
    double I = 1.0;
    switch (law) {
    case GCMC_LD_LINEAR: I = 1.0 - c[0] * x; break;
    case GCMC_LD_QUADRATIC: I = 1.0 - c[0] * x - c[1] * x * x; break;
    case GCMC_LD_SQRT: I = 1.0 - c[0] * x - c[1] * (1.0 - std::sqrt(mu)); break;
    case GCMC_LD_LOG: I = 1.0 - c[0] * x - c[1] * (mu > 0.0 ? mu * std::log(mu) : 0.0); break;
    case GCMC_LD_POWER2: I = 1.0 - c[0] * (1.0 - std::pow(mu, c[1])); break;
    case GCMC_LD_CLARET4:
        for (int k = 1; k <= 4; ++k) I -= c[k - 1] * (1.0 - std::pow(mu, 0.5 * k));
        break;
    default: break;
    }
    return I;
}

// the law as packets use it: negative values (bad coefficients) count as 0
static double limb_host(int law, const double *c, double mu)
{
    const double I = limb_raw(law, c, mu);
    return I > 0.0 ? I : 0.0;
}

// disk average 2 int_0^1 mu I(mu) dmu of a law, in closed form where the law stays non-negative
// (Gauss-Legendre on [0, 1] in sqrt(mu) otherwise, where clipping at 0 makes the integrand kinked)
static double limb_norm(int law, const double *c)
{
    bool nonneg = true;
    for (int t = 0; t <= 1000 && nonneg; ++t) nonneg = limb_raw(law, c, t / 1000.0) >= 0.0;
    if (nonneg) {
        switch (law) {
        case GCMC_LD_LINEAR: return 1.0 - c[0] / 3.0;
        case GCMC_LD_QUADRATIC: return 1.0 - c[0] / 3.0 - c[1] / 6.0;
        case GCMC_LD_SQRT: return 1.0 - c[0] / 3.0 - c[1] / 5.0;
        case GCMC_LD_LOG: return 1.0 - c[0] / 3.0 + 2.0 * c[1] / 9.0;
        case GCMC_LD_POWER2: return 1.0 - c[0] * c[1] / (c[1] + 2.0);
        case GCMC_LD_CLARET4: {
            double n = 1.0;
            for (int k = 1; k <= 4; ++k) n -= c[k - 1] * k / (k + 4.0);
            return n;
        }
        default: return 1.0;
        }
    }
    // composite midpoint rule in t = sqrt(mu): 2 int mu I dmu = 4 int t^3 I(t^2) dt
    const int n = 200000;
    double sum = 0.0;
    for (int i = 0; i < n; ++i) {
        const double t = (i + 0.5) / n;
        sum += 4.0 * t * t * t * limb_host(law, c, t * t);
    }
    return sum / n;
}

gcmc_status gcmc_transit(gcmc_ctx *ctx, int grid_id, int source_id, const double *tally, int64_t n_packets,
                         gcmc_transit_obs *out)
{
    if (!ctx || !tally || !out) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    if (grid_id < 0 || grid_id >= (int)ctx->grids.size()) return fail(ctx, GCMC_ERR_ARG, "bad grid_id");
    if (source_id < 0 || source_id >= (int)ctx->sources.size()) return fail(ctx, GCMC_ERR_ARG, "bad source_id");
    if (n_packets <= 0) return fail(ctx, GCMC_ERR_ARG, "n_packets must be positive");
    std::memset(out, 0, sizeof(*out));
    const gcmc_source_desc &s = ctx->sources[source_id];
    const double R0 = ctx->grids[grid_id].dg.R0, Rt = ctx->grids[grid_id].dg.Rtoa;
    const double k = (Rt - R0) / (double)n_packets * Rt;
    out->I_p_direct = k * tally[0];
    out->I_p_scattered = s.trans_scatter ? k * tally[1] : 0.0;
    const double Rs = s.star_radius, a = s.star_dist;
    out->omega_star = (a > Rs && Rs > 0.0) ? 2.0 * PI * (1.0 - std::sqrt(1.0 - (Rs / a) * (Rs / a))) : 0.0;
    out->I_p = out->I_p_direct - out->omega_star * out->I_p_scattered;
    out->w_core = 1.0;
    out->n_ld = 1.0;
    if (s.ld_law != GCMC_LD_NONE) {
        const double q = (s.transit_xy[0] * s.transit_xy[0] + s.transit_xy[1] * s.transit_xy[1]) / (Rs * Rs);
        out->w_core = q < 1.0 ? limb_host(s.ld_law, s.ld_coef, std::sqrt(1.0 - q)) : 0.0;
        out->n_ld = limb_norm(s.ld_law, s.ld_coef);
    }
    out->area = out->w_core * R0 * R0 + 2.0 * out->I_p;
    out->depth = Rs > 0.0 ? out->area / (Rs * Rs * out->n_ld) : 0.0;
    return GCMC_OK;
}

gcmc_status gcmc_release_grid(gcmc_ctx *ctx, int grid_id)
{
    if (!ctx || grid_id < 0 || grid_id >= (int)ctx->grids.size() || !ctx->grids[grid_id].dg.r)
        return fail(ctx, GCMC_ERR_ARG, "unknown or released grid");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    for (size_t o = 0; o < ctx->opacs.size(); ++o)
        if (ctx->opacs[o].grid == grid_id && !ctx->opacs[o].owned.empty()) gcmc_release_opacity(ctx, (int)o);
    GridH &G = ctx->grids[grid_id];
    for (void *p : G.owned) dfree(ctx, p);
    G.owned.clear();
    std::memset(&G.dg, 0, sizeof(G.dg));
    return GCMC_OK;
}

gcmc_status gcmc_release_opacity(gcmc_ctx *ctx, int opac_id)
{
    if (!ctx || opac_id < 0 || opac_id >= (int)ctx->opacs.size() || ctx->opacs[opac_id].owned.empty())
        return fail(ctx, GCMC_ERR_ARG, "unknown or released opacity");
    cudaSetDevice(ctx->device);
    cudaStreamSynchronize(ctx->stream);
    OpacH &O = ctx->opacs[opac_id];
    for (void *p : O.owned) dfree(ctx, p);
    O.owned.clear();
    O.grid = -1;
    return GCMC_OK;
}

gcmc_status gcmc_set_profiling(gcmc_ctx *ctx, int on)
{
    if (!ctx) return GCMC_ERR_ARG;
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    ctx->prof_ev.clear();
    ctx->prof = on != 0;
    return GCMC_OK;
}

gcmc_status gcmc_get_profile(gcmc_ctx *ctx, double *prep_ms, double *transport_ms, int64_t *transport_launches)
{
    if (!ctx) return GCMC_ERR_ARG;
    double a = 0.0, b = 0.0;
    int64_t n = 0;
    for (size_t q = 0; q + 3 <= ctx->prof_ev.size(); q += 3) {
        float x = 0.0f, y = 0.0f;
        if (cudaEventSynchronize(ctx->prof_ev[q + 2]) != cudaSuccess) return cuda_fail(ctx, cudaGetLastError(), "profile");
        cudaEventElapsedTime(&x, ctx->prof_ev[q], ctx->prof_ev[q + 1]);
        cudaEventElapsedTime(&y, ctx->prof_ev[q + 1], ctx->prof_ev[q + 2]);
        a += x;
        b += y;
        ++n;
    }
    for (cudaEvent_t e : ctx->prof_ev) cudaEventDestroy(e);
    ctx->prof_ev.clear();
    if (prep_ms) *prep_ms = a;
    if (transport_ms) *transport_ms = b;
    if (transport_launches) *transport_launches = n;
    return GCMC_OK;
}

int64_t gcmc_kernel_launches(void) { return (int64_t)g_launches.load(); }

gcmc_status gcmc_gather_bench(gcmc_ctx *ctx, int64_t n_records, int record_bytes, int64_t n_gathers, double *rate)
{
    if (!ctx || !rate || n_records < 1 || n_records > ((int64_t)1 << 32) - 1 || (record_bytes != 4 && record_bytes != 16) ||
        n_gathers < 1)
        return fail(ctx, GCMC_ERR_ARG, "gather bench arguments");
    cudaSetDevice(ctx->device);
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, ctx->device);
    const int threads = 256, blocks = nsm * 8;
    const int64_t per = std::max<int64_t>(1, n_gathers / ((int64_t)threads * blocks));
    void *tab = dalloc(ctx, (size_t)n_records * record_bytes);
    float *sink = (float *)dalloc(ctx, (size_t)threads * blocks * sizeof(float));
    if (!tab || !sink) {
        dfree(ctx, tab);
        dfree(ctx, sink);
        return fail(ctx, GCMC_ERR_OOM, "gather bench buffers");
    }
    cudaError_t e = cudaMemsetAsync(tab, 0x3c, (size_t)n_records * record_bytes, ctx->stream);
    cudaEvent_t a = nullptr, b = nullptr;
    cudaEventCreate(&a);
    cudaEventCreate(&b);
    if (e == cudaSuccess) e = gather_bench(tab, n_records, record_bytes, std::max<int64_t>(1, per / 8), blocks, threads, sink, ctx->stream);
    cudaEventRecord(a, ctx->stream);
    if (e == cudaSuccess) e = gather_bench(tab, n_records, record_bytes, per, blocks, threads, sink, ctx->stream);
    cudaEventRecord(b, ctx->stream);
    if (e == cudaSuccess) e = cudaEventSynchronize(b);
    float ms = 0.0f;
    if (e == cudaSuccess) cudaEventElapsedTime(&ms, a, b);
    cudaEventDestroy(a);
    cudaEventDestroy(b);
    dfree(ctx, tab);
    dfree(ctx, sink);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "gather bench");
    *rate = (double)per * threads * blocks / (ms * 1e-3);
    return GCMC_OK;
}

gcmc_status gcmc_selftest_philox(gcmc_ctx *ctx, const uint32_t *ctr, const uint32_t *key, int n, uint32_t *out_lib,
                                 uint32_t *out_curand)
{
    if (!ctx || n < 0 || (n > 0 && (!ctr || !key || !out_lib || !out_curand))) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    if (n == 0) return GCMC_OK;
    cudaSetDevice(ctx->device);
    uint32_t *d = (uint32_t *)dalloc(ctx, (size_t)n * 14 * sizeof(uint32_t));
    if (!d) return fail(ctx, GCMC_ERR_OOM, "selftest");
    uint32_t *dc = d, *dk = d + 4 * n, *dl = d + 6 * n, *du = d + 10 * n;
    cudaError_t e = cudaMemcpyAsync(dc, ctr, (size_t)n * 16, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(dk, key, (size_t)n * 8, cudaMemcpyHostToDevice, ctx->stream);
    if (e == cudaSuccess) e = selftest_philox(dc, dk, n, dl, du, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_lib, dl, (size_t)n * 16, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaMemcpyAsync(out_curand, du, (size_t)n * 16, cudaMemcpyDeviceToHost, ctx->stream);
    if (e == cudaSuccess) e = cudaStreamSynchronize(ctx->stream);
    dfree(ctx, d);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "philox selftest");
    return GCMC_OK;
}

}  // extern "C"

// ==================================================================== serving (continuous batching)
// A server owns two streams of its context: the serving kernel runs on one and never ends while
// there is published work; cell tables of newly admitted jobs are built on the other, beside it.
// Jobs wait in a host queue until a completion slot and their workspace fit (admission by HBM
// footprint), are prepared, and are published to the running kernel through host-mapped memory in
// admission order.  Completion records come back through host-mapped memory as well.
// per slot: the job records, then the initial value of the slot's claim counter
constexpr size_t SERVE_STAGE_BYTES = (sizeof(PrepJob) + sizeof(DevJob) + 8 + 255) & ~(size_t)255;

struct gcmc_server {
    struct Job {
        uint64_t ticket = 0;
        gcmc_job job{};
        int slot = -1;
        uint64_t seg = 0;
        uint32_t gen = 0;
        void *ws = nullptr;
        size_t bytes = 0;
        cudaEvent_t prepped = nullptr;
        int n_obs = 0;
        int64_t n_items = 0;
        const DevJob *djob = nullptr;
        bool published = false;
        bool ext = false;             // needs the kernel variant with the optional physics
        double t[4] = {0, 0, 0, 0};   // submitted, admitted, published, completed (s since creation)
    };
    struct Result {
        double tally[MAX_OBS];
        gcmc_stats st;
        double t[4];
    };
    std::chrono::steady_clock::time_point t0 = std::chrono::steady_clock::now();
    double now() const { return std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count(); }
    gcmc_ctx *ctx = nullptr;
    gcmc_server_cfg cfg{};
    cudaStream_t s_serve = nullptr, s_prep = nullptr;
    ServeCtl *ctl = nullptr;          // host-mapped (host pointers; the device sees the same addresses)
    ServeSeg *ring = nullptr;
    ServeDone *done = nullptr;
    char *stage_h = nullptr;          // pinned, one job-record staging area per completion slot
    cudaMemPool_t pool = nullptr;     // job workspaces (stream-ordered on the preparation stream)
    ServeQueue q{};
    unsigned long long *dstate = nullptr;
    std::deque<Job> pending;
    std::deque<Job> admitted;         // segment order
    std::map<uint64_t, Result> results;
    std::vector<int> free_slots;
    size_t bytes_in_use = 0;
    uint64_t next_ticket = 1, next_seg = 0, published = 0;
    uint32_t next_gen = 0;
    cudaEvent_t kdone = nullptr;
    bool kernel_started = false;
    bool kernel_ext = false;          // the running (or last) serving kernel carries the optional physics
    int tab_n = 0;
    int64_t kernel_launches = 0, completed = 0;
    int grid_blocks = 0;
};

namespace {

void server_free(gcmc_server *sv)
{
    if (sv->kdone) cudaEventDestroy(sv->kdone);
    for (auto *dq : {&sv->pending, &sv->admitted})
        for (auto &j : *dq) {
            if (j.prepped) cudaEventDestroy(j.prepped);
            if (j.ws) cudaFree(j.ws);
        }
    if (sv->dstate) cudaFree(sv->dstate);
    if (sv->ctl) cudaFreeHost(sv->ctl);
    if (sv->ring) cudaFreeHost(sv->ring);
    if (sv->done) cudaFreeHost(sv->done);
    if (sv->stage_h) cudaFreeHost(sv->stage_h);
    if (sv->pool) cudaMemPoolDestroy(sv->pool);
    if (sv->s_serve) cudaStreamDestroy(sv->s_serve);
    if (sv->s_prep) cudaStreamDestroy(sv->s_prep);
    delete sv;
}

bool kernel_running(gcmc_server *sv)
{
    return sv->kernel_started && cudaEventQuery(sv->kdone) == cudaErrorNotReady;
}

// oldest published segment that has not completed (next_seg when none)
uint64_t oldest_open(const gcmc_server *sv)
{
    uint64_t o = sv->next_seg;
    for (const auto &j : sv->admitted)
        if (j.published) o = std::min(o, j.seg);
    return o;
}

gcmc_status server_admit(gcmc_server *sv)
{
    gcmc_ctx *ctx = sv->ctx;
    while (!sv->pending.empty() && !sv->free_slots.empty()) {
        gcmc_server::Job &j = sv->pending.front();
        Plan P;
        gcmc_status s = plan_run(ctx, &j.job, 1, sv->cfg.chunk, P);
        if (s) return s;
        if (sv->bytes_in_use + P.ws_bytes > sv->cfg.hbm_budget && sv->bytes_in_use > 0) break;   // wait for memory
        void *ws = nullptr;
        CK(cudaMallocFromPoolAsync(&ws, P.ws_bytes, sv->pool, sv->s_prep));
        cudaStream_t keep = ctx->stream;
        ctx->stream = sv->s_prep;
        const int slot = sv->free_slots.back();
        s = stage(ctx, P, (char *)ws, nullptr, sv->stage_h + (size_t)slot * SERVE_STAGE_BYTES);
        ctx->stream = keep;
        if (s) {
            cudaFreeAsync(ws, sv->s_prep);
            return s;
        }
        j.ws = ws;
        j.bytes = P.ws_bytes;
        j.slot = slot;
        sv->free_slots.pop_back();
        j.n_obs = P.jobs[0].n_tal;
        j.ext = (P.feat & FEAT_EXT) != 0;
        j.n_items = (j.job.n_packets + sv->cfg.chunk - 1) / sv->cfg.chunk;
        j.djob = reinterpret_cast<const DevJob *>((char *)ws + P.off_jobs);
        j.gen = (++sv->next_gen) & 0xFFFFFFu;
        unsigned long long *init = reinterpret_cast<unsigned long long *>(
            sv->stage_h + (size_t)slot * SERVE_STAGE_BYTES + sizeof(PrepJob) + sizeof(DevJob));
        *init = (unsigned long long)j.gen << SERVE_GEN_SHIFT;
        CK(cudaMemcpyAsync(sv->q.slot_next + slot, init, 8, cudaMemcpyHostToDevice, sv->s_prep));
        CK(cudaMemsetAsync(sv->q.slot_done + slot, 0, 8, sv->s_prep));
        CK(cudaEventCreateWithFlags(&j.prepped, cudaEventDisableTiming));
        CK(cudaEventRecord(j.prepped, sv->s_prep));
        j.t[1] = sv->now();
        sv->bytes_in_use += j.bytes;
        sv->admitted.push_back(j);
        sv->pending.pop_front();
    }
    return GCMC_OK;
}

// Jobs are published as soon as their cell tables are ready (a job's claim and completion counters
// belong to its slot, so the order of segments is free).  A ring entry is rewritten only when every
// segment older than half a ring has completed.
gcmc_status server_publish(gcmc_server *sv)
{
    gcmc_ctx *ctx = sv->ctx;
    bool any = false;
    const uint64_t oldest = oldest_open(sv);
    // Every request runs in its own kernel variant (with or without the optional physics), so that its
    // result does not depend on what it is served with: the two variants round some FP32 operations
    // differently.  While a ready request needs the other variant than the running kernel, nothing more
    // is published; the kernel drains and leaves, and the next launch takes the variant of the oldest
    // ready request (server_kick), publishing only requests of that variant.
    const bool running = kernel_running(sv);
    int variant = running ? (sv->kernel_ext ? 1 : 0) : -1;
    for (const auto &j : sv->admitted) {
        if (j.published || cudaEventQuery(j.prepped) != cudaSuccess) continue;
        if (variant < 0) variant = j.ext ? 1 : 0;            // oldest ready request chooses the next launch
        else if ((j.ext ? 1 : 0) != variant && running) return GCMC_OK;
    }
    for (auto &j : sv->admitted) {
        if (j.published) continue;
        if ((j.ext ? 1 : 0) != variant) continue;
        if (sv->next_seg - oldest >= SERVE_RING / 2) break;
        const cudaError_t e = cudaEventQuery(j.prepped);
        if (e == cudaErrorNotReady) continue;
        if (e != cudaSuccess) return cuda_fail(ctx, e, "cell tables of a served job");
        j.seg = sv->next_seg++;
        ServeSeg &g = sv->ring[j.seg % SERVE_RING];
        g.job = j.djob;
        g.n_items = j.n_items;
        g.slot = (uint32_t)j.slot;
        g.gen = j.gen;
        j.published = true;
        j.t[2] = sv->now();
        sv->published = j.seg + 1;
        any = true;
    }
    if (any) __atomic_store_n(&sv->ctl->published, sv->published, __ATOMIC_RELEASE);
    return GCMC_OK;
}

gcmc_status server_collect(gcmc_server *sv, uint64_t *done_tickets, int cap, int *n_done)
{
    const unsigned err = __atomic_load_n(&sv->ctl->err, __ATOMIC_ACQUIRE);
    if (err & 1u) return fail(sv->ctx, GCMC_ERR_CUDA, "serving kernel: a work claim met a reused slot");
    if (err & 2u) return fail(sv->ctx, GCMC_ERR_TIMEOUT, "serving kernel: a warp waited past its idle cap");
    int nd = 0;
    for (auto it = sv->admitted.begin(); it != sv->admitted.end();) {
        gcmc_server::Job &j = *it;
        if (!j.published || __atomic_load_n(&sv->done[j.slot].seq, __ATOMIC_ACQUIRE) != j.seg + 1) {
            ++it;
            continue;
        }
        const ServeDone &d = sv->done[j.slot];
        gcmc_server::Result r;
        unpack(d.acc, d.info, j.n_obs, r.tally, &r.st);
        j.t[3] = sv->now();
        std::memcpy(r.t, j.t, sizeof(r.t));
        sv->results[j.ticket] = r;
        if (done_tickets && nd < cap) done_tickets[nd] = j.ticket;
        ++nd;
        cudaFreeAsync(j.ws, sv->s_prep);
        cudaEventDestroy(j.prepped);
        sv->bytes_in_use -= j.bytes;
        sv->free_slots.push_back(j.slot);
        ++sv->completed;
        it = sv->admitted.erase(it);
    }
    if (n_done) *n_done = nd;
    return GCMC_OK;
}

gcmc_status server_kick(gcmc_server *sv)
{
    gcmc_ctx *ctx = sv->ctx;
    bool open = false;
    for (const auto &j : sv->admitted)
        if (j.published) {
            open = true;
            break;
        }
    if (!open || kernel_running(sv)) return GCMC_OK;
    bool ext = false;   // the variant: with the optional physics when an open job needs it
    for (const auto &j : sv->admitted)
        if (j.published && j.ext) ext = true;
    const int idle_polls = sv->cfg.idle_us > 0 ? sv->cfg.idle_us : 2000;
    // a fresh launch: no warp idle, not leaving (stream-ordered after the previous launch)
    CK(cudaMemsetAsync(sv->q.n_idle, 0, 16, sv->s_serve));
    cudaError_t e = launch_serve(ext, ctx->d_grids, sv->q, sv->cfg.block, sv->cfg.blocks_per_sm, sv->cfg.chunk, sv->cfg.interval,
                                 sv->cfg.refill_min, sv->tab_n, idle_polls, &sv->grid_blocks, sv->s_serve);
    if (e != cudaSuccess) return cuda_fail(ctx, e, "serving kernel launch");
    CK(cudaEventRecord(sv->kdone, sv->s_serve));
    sv->kernel_started = true;
    sv->kernel_ext = ext;
    ++sv->kernel_launches;
    return GCMC_OK;
}

}  // namespace

extern "C" {

gcmc_status gcmc_server_create(gcmc_ctx *ctx, const gcmc_server_cfg *cfg, gcmc_server **out)
{
    if (!ctx || !out) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    *out = nullptr;
    cudaSetDevice(ctx->device);
    gcmc_server *sv = new gcmc_server();
    sv->ctx = ctx;
    if (cfg) sv->cfg = *cfg;
    gcmc_server_cfg &c = sv->cfg;
    if (c.block == 0) c.block = 128;
    if (c.chunk <= 0) c.chunk = 256;
    if (c.interval <= 0) c.interval = 4;
    if (c.refill_min <= 0) c.refill_min = 8;
    if (c.max_jobs <= 0) c.max_jobs = 1024;
    if (c.hbm_budget == 0) c.hbm_budget = (uint64_t)8 << 30;
    if (c.block != 128 || c.chunk % 32 || c.max_jobs > (int)(SERVE_RING / 2)) {
        delete sv;
        return fail(ctx, GCMC_ERR_ARG, "server: block must be 128, chunk a multiple of 32, max_jobs <= 32768");
    }
    for (const auto &g : ctx->grids)
        if (g.dg.r) sv->tab_n = std::max(sv->tab_n, tab_entries(g.dg.nlon, g.dg.nlat, g.dg.nr));
    if (sv->tab_n == 0) {
        delete sv;
        return fail(ctx, GCMC_ERR_ARG, "server: upload the grids first");
    }
    cudaError_t e = cudaStreamCreateWithFlags(&sv->s_serve, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaStreamCreateWithFlags(&sv->s_prep, cudaStreamNonBlocking);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&sv->ctl, sizeof(ServeCtl), cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&sv->ring, sizeof(ServeSeg) * SERVE_RING, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaHostAlloc((void **)&sv->done, sizeof(ServeDone) * c.max_jobs, cudaHostAllocMapped);
    if (e == cudaSuccess) e = cudaMallocHost((void **)&sv->stage_h, (size_t)SERVE_STAGE_BYTES * c.max_jobs);
    if (e == cudaSuccess) e = cudaMalloc(&sv->dstate, 8 * (3 + 2 * (size_t)c.max_jobs));
    if (e == cudaSuccess) e = cudaMemset(sv->dstate, 0, 8 * (3 + 2 * (size_t)c.max_jobs));
    if (e == cudaSuccess) e = cudaEventCreateWithFlags(&sv->kdone, cudaEventDisableTiming);
    if (e == cudaSuccess) {
        // a pool of its own that keeps freed workspace mapped (no release back to the driver)
        cudaMemPoolProps props{};
        props.allocType = cudaMemAllocationTypePinned;
        props.location.type = cudaMemLocationTypeDevice;
        props.location.id = ctx->device;
        e = cudaMemPoolCreate(&sv->pool, &props);
        uint64_t keep = ~0ull;
        if (e == cudaSuccess) e = cudaMemPoolSetAttribute(sv->pool, cudaMemPoolAttrReleaseThreshold, &keep);
    }
    ServeCtl *dctl = nullptr;
    ServeSeg *dring = nullptr;
    ServeDone *ddone = nullptr;
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&dctl, sv->ctl, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&dring, sv->ring, 0);
    if (e == cudaSuccess) e = cudaHostGetDevicePointer((void **)&ddone, sv->done, 0);
    if (e != cudaSuccess) {
        server_free(sv);
        return cuda_fail(ctx, e, "server create");
    }
    std::memset(sv->ctl, 0, sizeof(ServeCtl));
    std::memset(sv->ring, 0, sizeof(ServeSeg) * SERVE_RING);
    std::memset(sv->done, 0, sizeof(ServeDone) * c.max_jobs);
    sv->q.ctl = dctl;
    sv->q.ring = dring;
    sv->q.done = ddone;
    sv->q.cur_seg = sv->dstate;
    sv->q.n_idle = sv->dstate + 1;
    sv->q.exiting = sv->dstate + 2;
    sv->q.slot_next = sv->dstate + 3;
    sv->q.slot_done = sv->dstate + 3 + c.max_jobs;
    for (int s = c.max_jobs - 1; s >= 0; --s) sv->free_slots.push_back(s);
    *out = sv;
    return GCMC_OK;
}

gcmc_status gcmc_server_submit(gcmc_server *sv, const gcmc_job *job, uint64_t *ticket)
{
    if (!sv || !job || !ticket) return GCMC_ERR_ARG;
    gcmc_ctx *ctx = sv->ctx;
    gcmc_status s = check_job(ctx, *job);
    if (s) return s;
    if (job->n_packets < 1) return fail(ctx, GCMC_ERR_ARG, "a served job needs n_packets >= 1");
    if (ctx->sources[job->source_id].precision == GCMC_FP64) return fail(ctx, GCMC_ERR_ARG, "the server runs FP32 jobs");
    if (job->mode == GCMC_EMISSION && job->g_idx < 0)
        return fail(ctx, GCMC_ERR_ARG, "band jobs are not served: submit one job per g-ordinate");
    const DevGrid &g = ctx->grids[job->grid_id].dg;
    if (tab_entries(g.nlon, g.nlat, g.nr) > sv->tab_n)
        return fail(ctx, GCMC_ERR_ARG, "grid larger than every grid present when the server was created");
    gcmc_server::Job j;
    j.ticket = sv->next_ticket++;
    j.job = *job;
    j.t[0] = sv->now();
    sv->pending.push_back(j);
    *ticket = j.ticket;
    return GCMC_OK;
}

gcmc_status gcmc_server_progress(gcmc_server *sv, uint64_t *done_tickets, int cap, int *n_done)
{
    if (!sv) return GCMC_ERR_ARG;
    cudaSetDevice(sv->ctx->device);
    gcmc_status s = server_collect(sv, done_tickets, cap, n_done);
    if (!s) s = server_admit(sv);
    if (!s) s = server_publish(sv);
    if (!s) s = server_kick(sv);
    return s;
}

gcmc_status gcmc_server_result(gcmc_server *sv, uint64_t ticket, double *tallies_out, gcmc_stats *stats_out)
{
    if (!sv) return GCMC_ERR_ARG;
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) return GCMC_ERR_NOT_READY;
    if (tallies_out) std::memcpy(tallies_out, it->second.tally, sizeof(it->second.tally));
    if (stats_out) *stats_out = it->second.st;
    sv->results.erase(it);
    return GCMC_OK;
}

gcmc_status gcmc_server_times(gcmc_server *sv, uint64_t ticket, double *t4)
{
    if (!sv || !t4) return GCMC_ERR_ARG;
    auto it = sv->results.find(ticket);
    if (it == sv->results.end()) return GCMC_ERR_NOT_READY;
    std::memcpy(t4, it->second.t, sizeof(it->second.t));
    return GCMC_OK;
}

gcmc_status gcmc_server_query(gcmc_server *sv, gcmc_server_stats *st)
{
    if (!sv || !st) return GCMC_ERR_ARG;
    std::memset(st, 0, sizeof(*st));
    st->pending = (int64_t)sv->pending.size();
    st->admitted = (int64_t)sv->admitted.size();
    st->completed = sv->completed;
    st->bytes_in_use = sv->bytes_in_use;
    st->kernel_launches = sv->kernel_launches;
    st->kernel_running = kernel_running(sv) ? 1 : 0;
    st->grid_blocks = sv->grid_blocks;
    return GCMC_OK;
}

gcmc_status gcmc_server_destroy(gcmc_server *sv, double timeout_s)
{
    if (!sv) return GCMC_ERR_ARG;
    gcmc_ctx *ctx = sv->ctx;
    cudaSetDevice(ctx->device);
    // published work finishes first; the kernel leaves when it finds the queue empty and stop set
    __atomic_store_n(&sv->ctl->stop, 1u, __ATOMIC_RELEASE);
    gcmc_status s = GCMC_OK;
    if (sv->kernel_started) {
        const auto t0 = std::chrono::steady_clock::now();
        for (;;) {
            const cudaError_t e = cudaEventQuery(sv->kdone);
            if (e == cudaSuccess) break;
            if (e != cudaErrorNotReady) {
                s = cuda_fail(ctx, e, "serving kernel");
                break;
            }
            if (std::chrono::duration<double>(std::chrono::steady_clock::now() - t0).count() > timeout_s) {
                // the kernel is still draining published work: leave everything allocated
                return fail(ctx, GCMC_ERR_TIMEOUT, "serving kernel still running at destroy");
            }
            std::this_thread::sleep_for(std::chrono::microseconds(200));
        }
    }
    cudaStreamSynchronize(sv->s_prep);
    server_free(sv);
    return s;
}

}  // extern "C"

// ==================================================================== captured batches (CUDA graphs)
// A batch planned once and captured, with its cell-table kernels, the persistent transport launch and
// the conversion of the tallies, into one CUDA graph that replays on the context's stream.  The graph
// owns its workspace and its pinned job-record staging; replays recompute everything (cell tables
// included) from the resident grids and opacities.
struct gcmc_graph {
    gcmc_ctx *ctx = nullptr;
    Plan P;
    void *ws = nullptr;
    char *stage_h = nullptr;
    double *d_tally = nullptr;        // [n_jobs][MAX_OBS]
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
    int n_jobs = 0;
    long long kernels = 0;            // kernels in the graph (counted while capturing)
};

namespace {
void graph_free(gcmc_graph *g)
{
    if (g->exec) cudaGraphExecDestroy(g->exec);
    if (g->graph) cudaGraphDestroy(g->graph);
    if (g->stage_h) cudaFreeHost(g->stage_h);
    dfree(g->ctx, g->ws);
    dfree(g->ctx, g->d_tally);
    delete g;
}
}  // namespace

extern "C" {

gcmc_status gcmc_graph_create(gcmc_ctx *ctx, const gcmc_job *jobs, int n_jobs, const gcmc_launch_cfg *cfg,
                              gcmc_graph **out)
{
    if (!ctx || !jobs || !out) return fail(ctx, GCMC_ERR_ARG, "NULL argument");
    *out = nullptr;
    cudaSetDevice(ctx->device);
    if (!ctx->stream) return fail(ctx, GCMC_ERR_ARG, "capture needs a non-default stream (gcmc_set_stream)");
    const int chunk = cfg && cfg->chunk > 0 ? cfg->chunk : 1024;
    gcmc_graph *g = new gcmc_graph();
    g->ctx = ctx;
    g->n_jobs = n_jobs;
    gcmc_status s = plan_run(ctx, jobs, n_jobs, chunk, g->P);
    if (s) {
        delete g;
        return s;
    }
    Plan &P = g->P;
    const int prec = P.jobs[0].precision;
    for (const DevJob &d : P.jobs)
        if (d.precision != prec) {
            delete g;
            return fail(ctx, GCMC_ERR_ARG, "a batch runs in one precision");
        }
    g->ws = dalloc(ctx, P.ws_bytes);
    g->d_tally = (double *)dalloc(ctx, (size_t)n_jobs * MAX_OBS * sizeof(double));
    if (!g->ws || !g->d_tally ||
        cudaMallocHost((void **)&g->stage_h, P.prep.size() * sizeof(PrepJob) + n_jobs * sizeof(DevJob)) != cudaSuccess) {
        graph_free(g);
        return fail(ctx, GCMC_ERR_OOM, "graph workspace");
    }
    char *base = (char *)g->ws;
    const long long l0 = g_launches.load();
    cudaError_t e = cudaStreamBeginCapture(ctx->stream, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) {
        graph_free(g);
        return cuda_fail(ctx, e, "begin capture");
    }
    s = stage(ctx, P, base, nullptr, g->stage_h);
    if (!s) {
        const DevJob *dj = reinterpret_cast<const DevJob *>(base + P.off_jobs);
        e = launch_persistent(prec, P.scatter, P.feat, ctx->d_grids, dj, n_jobs, P.total_items, chunk, cfg ? cfg->block : 0,
                              cfg ? cfg->blocks_per_sm : 0, cfg && cfg->interval > 0 ? cfg->interval : 1,
                              cfg && cfg->refill_min > 0 ? cfg->refill_min : 16, P.one_grid, P.tab_n,
                              reinterpret_cast<unsigned long long *>(base + P.off_work), ctx->stream);
        if (e == cudaSuccess) {
            count_launch(1);
            k_acc_to_tallies<<<(n_jobs * MAX_OBS + 127) / 128, 128, 0, ctx->stream>>>(
                reinterpret_cast<unsigned long long *>(base + P.off_acc), n_jobs, g->d_tally);
            e = cudaGetLastError();
        }
    }
    const cudaError_t ec = cudaStreamEndCapture(ctx->stream, &g->graph);
    g->kernels = g_launches.load() - l0;
    g_launches.fetch_sub(g->kernels);   // captured, not launched: replays count them
    if (s || e != cudaSuccess || ec != cudaSuccess) {
        graph_free(g);
        if (s) return s;
        return cuda_fail(ctx, e != cudaSuccess ? e : ec, "capture");
    }
    e = cudaGraphInstantiate(&g->exec, g->graph, 0);
    if (e != cudaSuccess) {
        graph_free(g);
        return cuda_fail(ctx, e, "graph instantiate");
    }
    *out = g;
    return GCMC_OK;
}

gcmc_status gcmc_graph_launch(gcmc_graph *g, double *tallies_out)
{
    if (!g) return GCMC_ERR_ARG;
    gcmc_ctx *ctx = g->ctx;
    cudaSetDevice(ctx->device);
    count_launch((int)g->kernels);
    CK(cudaGraphLaunch(g->exec, ctx->stream));
    if (tallies_out)
        CK(cudaMemcpyAsync(tallies_out, g->d_tally, (size_t)g->n_jobs * MAX_OBS * sizeof(double), cudaMemcpyDeviceToDevice,
                           ctx->stream));
    return GCMC_OK;
}

gcmc_status gcmc_graph_read(gcmc_graph *g, double *tallies_out, gcmc_stats *stats_out)
{
    if (!g) return GCMC_ERR_ARG;
    gcmc_ctx *ctx = g->ctx;
    cudaSetDevice(ctx->device);
    return finish_run(ctx, g->P, (char *)g->ws, tallies_out, GCMC_MEM_HOST, stats_out, 1);
}

gcmc_status gcmc_graph_destroy(gcmc_graph *g)
{
    if (!g) return GCMC_ERR_ARG;
    cudaSetDevice(g->ctx->device);
    cudaStreamSynchronize(g->ctx->stream);
    graph_free(g);
    return GCMC_OK;
}

}  // extern "C"
