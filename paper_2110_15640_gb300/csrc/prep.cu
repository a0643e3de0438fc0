// prep.cu -- S1: per-job cell tables, computed on the device for every job of a launch.
//
//   albedo       alpha_ext = rho (k_abs + k_Ray) + a_cld q_cld, omega = alpha_sca / alpha_ext,
//                P_gas = rho k_Ray / alpha_sca (Sect. 3.6), HG g; FP64 arithmetic, stored as one
//                16-byte FP32 record per cell (32 bytes in FP64 runs).
//   emission     alpha = rho k(T, p) from the correlated-k table (bilinear in ln T, ln p of ln k),
//                L_i = 4 pi V_i alpha_i B_lambda(T_i) (Sect. 5.3), the tau_vert cut (Sect. 4.6),
//                hybrid pdf q_i = (1 - beta) L_i/L_tot + beta/N'_c and launch weight (L_i/L_tot)/q_i
//                (Sect. 4.3), and its cumulative sum in 64-bit fixed point (exact, monotone, flat
//                over excluded cells).  4 pi V B(T) is computed once per band (FP64); L_i, L_tot and
//                the fixed-point pdf are FP64.  FP64 runs compute alpha and the weights in FP64 term
//                by term; FP32 runs compute alpha in FP32 (~3e-7 relative) and FP32 weights, which is
//                what their march and tallies consume.
//   transmission per-cell v_LOS (Sect. 7), lambda_eff = lambda_0 (1 - v_LOS / c), cross-section
//                interpolated linearly in ln sigma between the bracketing table wavelengths and
//                bilinearly in (ln T, ln p); FP32 in FP32 runs (no integer decision depends on it).
#include <curand_philox4x32_x.h>

#include <algorithm>
#include <cstring>
#include <type_traits>

#include "internal.h"

namespace gcmc {

__device__ __forceinline__ void interp_idx(const double *grid, int n, double v, int &a, double &w)
{
    if (v <= grid[0]) {
        a = 0;
        w = 0.0;
        return;
    }
    if (v >= grid[n - 1]) {
        a = n - 2;
        w = 1.0;
        return;
    }
    int lo = 0, hi = n - 1;
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (grid[mid] <= v) lo = mid; else hi = mid;
    }
    a = lo;
    w = (log(v) - log(grid[lo])) / (log(grid[lo + 1]) - log(grid[lo]));
}

// ------------------------------------------------------------------ albedo
template <typename real>
__global__ void k_prep_albedo(DevGrid G, AlbDev op, const PrepJob *__restrict__ jobs)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= G.ncell) return;
    const PrepJob pj = jobs[blockIdx.y];
    const int l = pj.lam;
    const double rho = (double)G.rho[idx];
    const double ac = op.acld ? (double)op.acld[idx] * op.qcld[l] : 0.0;
    const double ray = rho * op.kray[l];
    const double ext = rho * (op.kabs[l] + op.kray[l]) + ac;
    const double sca = ray + op.wcld[l] * ac;
    const double om = ext > 0.0 ? sca / ext : 0.0;
    const double pg = sca > 0.0 ? ray / sca : 1.0;
    if (pj.alpha) reinterpret_cast<real *>(pj.alpha)[idx] = (real)ext;
    if constexpr (sizeof(real) == 4) {
        reinterpret_cast<float4 *>(pj.rec)[idx] = make_float4((float)ext, (float)om, (float)op.gcld[l], (float)pg);
    } else {
        Rec64 r;
        r.a = ext;
        r.w = om;
        r.g = op.gcld[l];
        r.pg = pg;
        reinterpret_cast<Rec64 *>(pj.rec)[idx] = r;
    }
}

std::atomic<long long> g_launches{0};

cudaError_t prep_albedo(int precision, const DevGrid *, const DevGrid &hg, const AlbDev &op, const PrepJob *djobs,
                        int njobs, cudaStream_t st)
{
    count_launch(1);
    dim3 grid((unsigned)((hg.ncell + PREP_BLOCK - 1) / PREP_BLOCK), (unsigned)njobs);
    if (precision == GCMC_FP64) k_prep_albedo<double><<<grid, PREP_BLOCK, 0, st>>>(hg, op, djobs);
    else k_prep_albedo<float><<<grid, PREP_BLOCK, 0, st>>>(hg, op, djobs);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ interpolation weights (T, p)
__global__ void k_tp_weights(DevGrid G, const double *Tg, int nT, const double *pg, int np, int2 *ab, double2 *w64,
                             float2 *w32)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= G.ncell) return;
    int a, b;
    double wT, wp;
    interp_idx(Tg, nT, (double)G.T[idx], a, wT);
    interp_idx(pg, np, (double)G.p[idx], b, wp);
    ab[idx] = make_int2(a, b);
    w64[idx] = make_double2(wT, wp);
    w32[idx] = make_float2((float)wT, (float)wp);
}

// ------------------------------------------------------------------ emission
// 4 pi V_i B_lambda(T_i) for every band centre (row b of vb), once per k-table upload
__global__ void k_emis_planck(DevGrid G, const double *__restrict__ lam, double *vb)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= G.ncell) return;
    const double l = lam[blockIdx.y];
    const double c1 = 2.0 * H_PLANCK * C_LIGHT * C_LIGHT / (l * l * l * l * l);
    const double x = H_PLANCK * C_LIGHT / (l * K_BOLTZ * (double)G.T[idx]);
    vb[(int64_t)blockIdx.y * G.ncell + idx] = 4.0 * PI * G.vol[idx] * (c1 / expm1(x));
}

cudaError_t ktable_cells(const DevGrid &hg, const double *lam_dev, int nb, int2 *ab, double2 *w64, float2 *w32, double *vb,
                         const KtabDev &kt, cudaStream_t st)
{
    count_launch(2);
    const unsigned nbk = (unsigned)((hg.ncell + PREP_BLOCK - 1) / PREP_BLOCK);
    k_tp_weights<<<nbk, PREP_BLOCK, 0, st>>>(hg, kt.Tg, kt.nT, kt.pg, kt.np, ab, w64, w32);
    k_emis_planck<<<dim3(nbk, (unsigned)nb), PREP_BLOCK, 0, st>>>(hg, lam_dev, vb);
    return cudaGetLastError();
}

constexpr int COL_BLOCK = 128;

int emis_col_blocks(const DevGrid &g) { return (int)(((int64_t)g.nlon * g.nlat + COL_BLOCK - 1) / COL_BLOCK); }

// One thread per (job, column), walking the column from the top: alpha = rho k(T, p), the tau_vert
// cut (a cell emits if the vertical optical depth above it is below tau_vert_max), L_i = 4 pi V_i
// B(T_i) alpha_i, and per-block partial sums of L and of the emitting-cell count (fixed order).
// Excluded cells get L = -1 in the scratch copy that the pdf kernel reads.
template <typename real>
__global__ void __launch_bounds__(COL_BLOCK) k_emis_column(DevGrid G, KtabDev kt, const PrepJob *__restrict__ jobs,
                                                           double tau_vert_max)
{
    extern __shared__ __align__(16) unsigned char col_smem[];
    real *s_dr = reinterpret_cast<real *>(col_smem);     // layer thicknesses [nr]
    __shared__ double red_s[COL_BLOCK / 32];
    __shared__ int red_c[COL_BLOCK / 32];
    for (int k = threadIdx.x; k < G.nr; k += blockDim.x) s_dr[k] = (real)(G.r[k + 1] - G.r[k]);
    __syncthreads();
    const PrepJob &pj = jobs[blockIdx.y];
    const int64_t ncol = (int64_t)G.nlon * G.nlat;
    const int64_t col = (int64_t)blockIdx.x * COL_BLOCK + threadIdx.x;
    double lsum = 0.0;
    int cnt = 0;
    if (col < ncol) {
        const double *__restrict__ vb = kt.vb + (int64_t)pj.lam * G.ncell;
        const int2 *__restrict__ ab = kt.ab;
        real *__restrict__ rec = reinterpret_cast<real *>(pj.rec);
        double *__restrict__ lb = reinterpret_cast<double *>(pj.cdf);
        double *__restrict__ lum = pj.lum;
        const int64_t slice = ((int64_t)pj.lam * kt.ng + pj.g) * kt.nT * kt.np;
        const real tmax = (real)tau_vert_max;
        real above = (real)0;
        for (int k = G.nr - 1; k >= 0; --k) {
            const int64_t idx = k * ncol + col;
            const int2 q = ab[idx];
            real alpha;
            if constexpr (sizeof(real) == 8) {
                const double2 ww = kt.w64[idx];
                const double wT = ww.x, wp = ww.y;
                const double *base = kt.lnk + slice;
                const double l00 = base[q.x * kt.np + q.y], l10 = base[(q.x + 1) * kt.np + q.y];
                const double l01 = base[q.x * kt.np + q.y + 1], l11 = base[(q.x + 1) * kt.np + q.y + 1];
                const double lk = (1 - wT) * (1 - wp) * l00 + wT * (1 - wp) * l10 + (1 - wT) * wp * l01 + wT * wp * l11;
                alpha = (double)G.rho[idx] * exp(lk);
            } else {
                const float2 ww = kt.w32[idx];
                const float4 nd = __ldg(kt.node_f + slice + q.x * kt.np + q.y);
                alpha = (G.rho[idx] * nd.x) * expf(fmaf(ww.x, fmaf(ww.y, nd.w, nd.y), ww.y * nd.z));
            }
            rec[idx] = alpha;
            const bool incl = above < tmax;
            above += alpha * s_dr[k];
            const double L = vb[idx] * (double)alpha;
            if (lum) lum[idx] = L;
            if (incl) {
                lb[idx] = L;
                lsum += L;
                ++cnt;
            } else {
                lb[idx] = -1.0;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lsum += __shfl_down_sync(0xffffffffu, lsum, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red_s[threadIdx.x >> 5] = lsum;
        red_c[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        int c = 0;
        for (int q = 0; q < COL_BLOCK / 32; ++q) {
            s += red_s[q];
            c += red_c[q];
        }
        pj.bsum[blockIdx.x] = s;
        pj.bcnt[blockIdx.x] = (double)c;
    }
}

// The same column walk for cells whose extinction is already in the job's table (Doppler-shifted
// cross-sections, Sect. 7): L_i = 4 pi V_i B_lambda(T_i) alpha_i with B at the job's wavelength.
template <typename real>
__global__ void __launch_bounds__(COL_BLOCK) k_emis_column_alpha(DevGrid G, const PrepJob *__restrict__ jobs,
                                                                 double tau_vert_max)
{
    extern __shared__ __align__(16) unsigned char col_smem[];
    real *s_dr = reinterpret_cast<real *>(col_smem);     // layer thicknesses [nr]
    __shared__ double red_s[COL_BLOCK / 32];
    __shared__ int red_c[COL_BLOCK / 32];
    for (int k = threadIdx.x; k < G.nr; k += blockDim.x) s_dr[k] = (real)(G.r[k + 1] - G.r[k]);
    __syncthreads();
    const PrepJob &pj = jobs[blockIdx.y];
    const int64_t ncol = (int64_t)G.nlon * G.nlat;
    const int64_t col = (int64_t)blockIdx.x * COL_BLOCK + threadIdx.x;
    double lsum = 0.0;
    int cnt = 0;
    if (col < ncol) {
        const real *__restrict__ rec = reinterpret_cast<const real *>(pj.rec);
        double *__restrict__ lb = reinterpret_cast<double *>(pj.cdf);
        double *__restrict__ lum = pj.lum;
        const double l = pj.lam_m;
        const double c1 = 2.0 * H_PLANCK * C_LIGHT * C_LIGHT / (l * l * l * l * l);
        const double hck = H_PLANCK * C_LIGHT / (l * K_BOLTZ);
        const real tmax = (real)tau_vert_max;
        real above = (real)0;
        for (int k = G.nr - 1; k >= 0; --k) {
            const int64_t idx = k * ncol + col;
            const real alpha = rec[idx];
            const bool incl = above < tmax;
            above += alpha * s_dr[k];
            // B_lambda(T_i) per cell and job: FP64 for FP64 runs; FP32 runs evaluate the exponential in FP32
            // (~1e-7 relative, below the FP32 extinction's own rounding), the sums stay FP64
            double B;
            if constexpr (sizeof(real) == 8) B = c1 / expm1(hck / (double)G.T[idx]);
            else B = (double)((float)c1 / expm1f((float)hck / G.T[idx]));
            const double L = 4.0 * PI * G.vol[idx] * B * (double)alpha;
            if (lum) lum[idx] = L;
            if (incl) {
                lb[idx] = L;
                lsum += L;
                ++cnt;
            } else {
                lb[idx] = -1.0;
            }
        }
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lsum += __shfl_down_sync(0xffffffffu, lsum, o);
        cnt += __shfl_down_sync(0xffffffffu, cnt, o);
    }
    if ((threadIdx.x & 31) == 0) {
        red_s[threadIdx.x >> 5] = lsum;
        red_c[threadIdx.x >> 5] = cnt;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        double s = 0.0;
        int c = 0;
        for (int q = 0; q < COL_BLOCK / 32; ++q) {
            s += red_s[q];
            c += red_c[q];
        }
        pj.bsum[blockIdx.x] = s;
        pj.bcnt[blockIdx.x] = (double)c;
    }
}

// per-block sums of L over the emitting cells (L >= 0) and their count, for an L array given directly
// (the allocation-free entry point)
__global__ void k_emis_reduce(int64_t ncell, const PrepJob *__restrict__ jobs)
{
    __shared__ double ss[EMIS_SCAN_BLOCK / 32], sc[EMIS_SCAN_BLOCK / 32];
    const PrepJob pj = jobs[blockIdx.y];
    const int64_t idx = (int64_t)blockIdx.x * EMIS_SCAN_BLOCK + threadIdx.x;
    const double *lb = reinterpret_cast<const double *>(pj.cdf);
    double L = idx < ncell ? lb[idx] : -1.0;
    double v = L >= 0.0 ? L : 0.0, c = L >= 0.0 ? 1.0 : 0.0;
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        v += __shfl_down_sync(0xffffffffu, v, o);
        c += __shfl_down_sync(0xffffffffu, c, o);
    }
    if ((threadIdx.x & 31) == 0) {
        ss[threadIdx.x >> 5] = v;
        sc[threadIdx.x >> 5] = c;
    }
    __syncthreads();
    if (threadIdx.x < 32) {
        constexpr int NW = EMIS_SCAN_BLOCK / 32;
        v = threadIdx.x < NW ? ss[threadIdx.x] : 0.0;
        c = threadIdx.x < NW ? sc[threadIdx.x] : 0.0;
#pragma unroll
        for (int o = 16; o; o >>= 1) {
            v += __shfl_down_sync(0xffffffffu, v, o);
            c += __shfl_down_sync(0xffffffffu, c, o);
        }
        if (threadIdx.x == 0) {
            pj.bsum[blockIdx.x] = v;
            pj.bcnt[blockIdx.x] = c;
        }
    }
}

// The cumulative pdf is accumulated in 64-bit fixed point, Q_i = round(q_i 2^62) (sum <= 2^62 (1 + eps)):
// integer prefix sums are exact in any order, so the cumulative sum is monotone and exactly flat over
// cells with zero pdf, whatever the block and warp structure of the scan.
constexpr double CDF_FIX = 4611686018427387904.0;   // 2^62

// totals of the partial sums (fixed order) and the per-job constants of the hybrid pdf
// q_i = (1 - beta) L_i / L_tot + beta / n_incl (Sect. 4.3)
__global__ void k_emis_total(int nparts, const PrepJob *__restrict__ jobs, int njobs, double beta)
{
    const int jb = blockIdx.x * blockDim.x + threadIdx.x;
    if (jb >= njobs) return;
    const PrepJob pj = jobs[jb];
    double s = 0.0, c = 0.0;
    for (int b = 0; b < nparts; ++b) {
        s += pj.bsum[b];
        c += pj.bcnt[b];
    }
    double qa = 0.0, qb = 0.0, invl = 0.0, bn = 0.0;
    if (c > 0.0) {
        if (s > 0.0) {
            qa = (1.0 - beta) / s * CDF_FIX;
            qb = beta / c * CDF_FIX;
            invl = 1.0 / s;
            bn = beta / c;
        } else {
            qb = CDF_FIX / c;
        }
    }
    pj.info[INFO_LTOT] = s;
    pj.info[INFO_NINCL] = c;
    pj.info[INFO_QA] = qa;
    pj.info[INFO_QB] = qb;
    pj.info[INFO_INVL] = invl;
    pj.info[INFO_BN] = bn;
}

__device__ __forceinline__ long long warp_incl_scan_ll(long long v)
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int o = 1; o < 32; o <<= 1) {
        const long long t = __shfl_up_sync(0xffffffffu, v, o);
        if (lane >= o) v += t;
    }
    return v;
}

// hybrid pdf, launch weight (L_i / L_tot) / q_i and the per-block inclusive scan of the fixed-point pdf.
// FP64 weights follow the definition term by term; FP32 weights are p / ((1 - beta) p + beta / n) with
// p = L_i / L_tot rounded to FP32, and the fixed-point pdf is rint(QA L_i + QB) (one FP64 FMA).
template <typename WT>
__global__ void k_emis_pdf(int64_t ncell, const PrepJob *__restrict__ jobs, double beta)
{
    __shared__ long long ws[EMIS_SCAN_BLOCK / 32];
    const PrepJob &pj = jobs[blockIdx.y];
    const int64_t idx = (int64_t)blockIdx.x * EMIS_SCAN_BLOCK + threadIdx.x;
    long long Q = 0;
    WT wgt = (WT)0;
    if (idx < ncell) {
        const double L = reinterpret_cast<const double *>(pj.cdf)[idx];
        if constexpr (sizeof(WT) == 8) {
            const double Ltot = pj.info[INFO_LTOT], nincl = pj.info[INFO_NINCL];
            if (L >= 0.0 && nincl > 0.0) {
                double q;
                if (Ltot > 0.0) {
                    q = (1.0 - beta) * L / Ltot + beta / nincl;
                    wgt = q > 0.0 ? (L / Ltot) / q : 0.0;
                } else {
                    q = 1.0 / nincl;
                }
                Q = __double2ll_rn(q * CDF_FIX);
            }
        } else {
            if (L >= 0.0) {
                Q = __double2ll_rn(fma(pj.info[INFO_QA], L, pj.info[INFO_QB]));
                const float p = (float)(L * pj.info[INFO_INVL]);
                const float qf = fmaf((float)(1.0 - beta), p, (float)pj.info[INFO_BN]);
                wgt = qf > 0.0f ? p / qf : 0.0f;
            }
        }
    }
    long long s = warp_incl_scan_ll(Q);
    if ((threadIdx.x & 31) == 31) ws[threadIdx.x >> 5] = s;
    __syncthreads();
    if (threadIdx.x < 32) {
        constexpr int NW = EMIS_SCAN_BLOCK / 32;
        const long long t = warp_incl_scan_ll(threadIdx.x < NW ? ws[threadIdx.x] : 0ll);
        if (threadIdx.x < NW) ws[threadIdx.x] = t;
    }
    __syncthreads();
    if (threadIdx.x >= 32) s += ws[(threadIdx.x >> 5) - 1];
    if (idx < ncell) {
        pj.cdf[idx] = s;     // within-block prefix until cdf_add
        reinterpret_cast<WT *>(pj.wcell)[idx] = wgt;
    }
    if (threadIdx.x == EMIS_SCAN_BLOCK - 1) reinterpret_cast<long long *>(pj.bsum)[blockIdx.x] = s;
}

// exclusive prefix of the per-block totals (one warp per job, 32 blocks per pass) and the job's total
__global__ void k_emis_scan_blocks(int nblk, const PrepJob *__restrict__ jobs, int njobs)
{
    const int jb = (int)((blockIdx.x * blockDim.x + threadIdx.x) >> 5);
    const int lane = threadIdx.x & 31;
    if (jb >= njobs) return;
    const PrepJob &pj = jobs[jb];
    const long long *bt = reinterpret_cast<const long long *>(pj.bsum);
    long long *off = reinterpret_cast<long long *>(pj.bcnt);
    long long run = 0;
    for (int b0 = 0; b0 < nblk; b0 += 32) {
        const int b = b0 + lane;
        const long long t = b < nblk ? bt[b] : 0ll;
        const long long inc = warp_incl_scan_ll(t);
        if (b < nblk) off[b] = run + inc - t;
        run += __shfl_sync(0xffffffffu, inc, 31);
    }
    if (lane == 0) {
        pj.info[INFO_CDFTOT] = (double)run / CDF_FIX;
        reinterpret_cast<long long *>(pj.info)[INFO_QTOT] = run;
    }
}

// block offsets added to the within-block prefixes: the fixed-point cumulative pdf itself (OUT =
// long long, what the launch searches) or its value as FP64 (OUT = double)
template <typename OUT>
__global__ void k_emis_cdf_add(int64_t ncell, const PrepJob *__restrict__ jobs)
{
    const PrepJob &pj = jobs[blockIdx.y];
    const int64_t idx = (int64_t)blockIdx.x * EMIS_SCAN_BLOCK + threadIdx.x;
    if (idx >= ncell) return;
    const long long v = pj.cdf[idx] + reinterpret_cast<const long long *>(pj.bcnt)[blockIdx.x];
    if constexpr (std::is_same<OUT, double>::value) reinterpret_cast<double *>(pj.cdf)[idx] = (double)v / CDF_FIX;
    else pj.cdf[idx] = v;
}

// One pass per job over its cells: the hybrid pdf and launch weights of k_emis_pdf and the fixed-point
// cumulative pdf, a block per job sweeping its cells in tiles of 4 cells per thread with the running
// total carried from tile to tile (the next tile's luminosities are loaded before the current tile is
// scanned), and the job's total into info.  The same integers as k_emis_pdf + k_emis_scan_blocks +
// k_emis_cdf_add (integer prefix sums are exact in any order) with one read of L_i and one write of the
// cumulative pdf and the weights per cell.
constexpr int EMIS_SWEEP_BLOCK = 1024;
constexpr int EMIS_SWEEP_TILE = 4 * EMIS_SWEEP_BLOCK;

// the 4 luminosities of cells i0 .. i0 + 3 (16-byte loads when vec), -1 past the last cell
__device__ __forceinline__ void emis_load4(const double *__restrict__ Lp, int64_t i0, int64_t ncell, bool vec, double L[4])
{
    if (vec && i0 + 3 < ncell) {
        const double2 a = *reinterpret_cast<const double2 *>(Lp + i0), b = *reinterpret_cast<const double2 *>(Lp + i0 + 2);
        L[0] = a.x;
        L[1] = a.y;
        L[2] = b.x;
        L[3] = b.y;
    } else {
#pragma unroll
        for (int q = 0; q < 4; ++q) L[q] = i0 + q < ncell ? Lp[i0 + q] : -1.0;
    }
}

template <typename WT>
__global__ void __launch_bounds__(EMIS_SWEEP_BLOCK) k_emis_sweep(int64_t ncell, const PrepJob *__restrict__ jobs,
                                                                 double beta)
{
    constexpr int NW = EMIS_SWEEP_BLOCK / 32;
    __shared__ long long ws[NW];
    const PrepJob &pj = jobs[blockIdx.x];
    const double *Lp = reinterpret_cast<const double *>(pj.cdf);   // L_i in place, read before written
    WT *wp = reinterpret_cast<WT *>(pj.wcell);
    // 16-byte loads and stores when every job array of this block is aligned for them
    const bool vec = ((reinterpret_cast<uintptr_t>(pj.cdf) | reinterpret_cast<uintptr_t>(pj.wcell)) & 15) == 0;
    const double Ltot = pj.info[INFO_LTOT], nincl = pj.info[INFO_NINCL];
    const double qa = pj.info[INFO_QA], qb = pj.info[INFO_QB], invl = pj.info[INFO_INVL];
    const float bn = (float)pj.info[INFO_BN], omb = (float)(1.0 - beta);
    const int lane = threadIdx.x & 31, warp = threadIdx.x >> 5;
    long long carry = 0;
    double L[4];
    emis_load4(Lp, 4 * (int64_t)threadIdx.x, ncell, vec, L);
    for (int64_t base = 0; base < ncell; base += EMIS_SWEEP_TILE) {
        const int64_t i0 = base + 4 * (int64_t)threadIdx.x;
        long long Q[4];
        WT w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            Q[q] = 0;
            w[q] = (WT)0;
            if constexpr (sizeof(WT) == 8) {
                if (L[q] >= 0.0 && nincl > 0.0) {
                    double qq;
                    if (Ltot > 0.0) {
                        qq = (1.0 - beta) * L[q] / Ltot + beta / nincl;
                        w[q] = qq > 0.0 ? (L[q] / Ltot) / qq : 0.0;
                    } else {
                        qq = 1.0 / nincl;
                    }
                    Q[q] = __double2ll_rn(qq * CDF_FIX);
                }
            } else {
                if (L[q] >= 0.0) {
                    Q[q] = __double2ll_rn(fma(qa, L[q], qb));
                    const float pp = (float)(L[q] * invl);
                    const float qf = fmaf(omb, pp, bn);
                    w[q] = qf > 0.0f ? pp / qf : 0.0f;
                }
            }
        }
        // the next tile's luminosities in flight while this one is scanned
        if (base + EMIS_SWEEP_TILE < ncell) emis_load4(Lp, i0 + EMIS_SWEEP_TILE, ncell, vec, L);
        const long long s1 = Q[0] + Q[1], s2 = s1 + Q[2], t = s2 + Q[3];
        const long long inc = warp_incl_scan_ll(t);
        if (lane == 31) ws[warp] = inc;
        __syncthreads();
        if (warp == 0) {
            const long long v = warp_incl_scan_ll(lane < NW ? ws[lane] : 0ll);
            if (lane < NW) ws[lane] = v;
        }
        __syncthreads();
        const long long pre = carry + (warp ? ws[warp - 1] : 0ll) + inc - t;
        const long long c[4] = {pre + Q[0], pre + s1, pre + s2, pre + t};
        if (vec && i0 + 3 < ncell) {
            *reinterpret_cast<longlong2 *>(pj.cdf + i0) = make_longlong2(c[0], c[1]);
            *reinterpret_cast<longlong2 *>(pj.cdf + i0 + 2) = make_longlong2(c[2], c[3]);
            if constexpr (sizeof(WT) == 8) {
                *reinterpret_cast<double2 *>(wp + i0) = make_double2(w[0], w[1]);
                *reinterpret_cast<double2 *>(wp + i0 + 2) = make_double2(w[2], w[3]);
            } else {
                *reinterpret_cast<float4 *>(wp + i0) = make_float4(w[0], w[1], w[2], w[3]);
            }
        } else {
#pragma unroll
            for (int q = 0; q < 4; ++q)
                if (i0 + q < ncell) {
                    pj.cdf[i0 + q] = c[q];
                    wp[i0 + q] = w[q];
                }
        }
        carry += ws[NW - 1];
        __syncthreads();     // ws is written again by the next tile
    }
    if (threadIdx.x == 0) {
        pj.info[INFO_CDFTOT] = (double)carry / CDF_FIX;
        reinterpret_cast<long long *>(pj.info)[INFO_QTOT] = carry;
    }
}

// the hybrid pdf, fixed-point CDF and launch weights from the column kernels' luminosities and sums
static cudaError_t emission_pdf(bool f64, const DevGrid &hg, const PrepJob *djobs, int njobs, int ncolb, double beta,
                                cudaStream_t st)
{
    k_emis_total<<<(njobs + 127) / 128, 128, 0, st>>>(ncolb, djobs, njobs, beta);
    // one sweep block per job keeps one SM busy per job: for batches that fill the GPU with jobs; fewer
    // jobs (a single job of the plain form or of the server) take the per-block pdf and scan, whose
    // blocks spread every job over the whole GPU
    int dev = 0, nsm = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (3 * njobs >= 2 * nsm) {
        count_launch(2);
        if (f64) k_emis_sweep<double><<<(unsigned)njobs, EMIS_SWEEP_BLOCK, 0, st>>>(hg.ncell, djobs, beta);
        else k_emis_sweep<float><<<(unsigned)njobs, EMIS_SWEEP_BLOCK, 0, st>>>(hg.ncell, djobs, beta);
        return cudaGetLastError();
    }
    count_launch(4);
    const int nblk = (int)((hg.ncell + EMIS_SCAN_BLOCK - 1) / EMIS_SCAN_BLOCK);
    const dim3 g3((unsigned)nblk, (unsigned)njobs);
    if (f64) k_emis_pdf<double><<<g3, EMIS_SCAN_BLOCK, 0, st>>>(hg.ncell, djobs, beta);
    else k_emis_pdf<float><<<g3, EMIS_SCAN_BLOCK, 0, st>>>(hg.ncell, djobs, beta);
    k_emis_scan_blocks<<<(njobs + 3) / 4, 128, 0, st>>>(nblk, djobs, njobs);
    k_emis_cdf_add<long long><<<g3, EMIS_SCAN_BLOCK, 0, st>>>(hg.ncell, djobs);
    return cudaGetLastError();
}

cudaError_t prep_emission(int precision, const DevGrid &hg, const KtabDev &kt, const PrepJob *djobs, int njobs,
                          double tau_vert_max, double beta, cudaStream_t st)
{
    count_launch(1);
    const bool f64 = precision == GCMC_FP64;
    const int ncolb = emis_col_blocks(hg);
    const dim3 gc((unsigned)ncolb, (unsigned)njobs);
    if (f64) k_emis_column<double><<<gc, COL_BLOCK, hg.nr * sizeof(double), st>>>(hg, kt, djobs, tau_vert_max);
    else k_emis_column<float><<<gc, COL_BLOCK, hg.nr * sizeof(float), st>>>(hg, kt, djobs, tau_vert_max);
    return emission_pdf(f64, hg, djobs, njobs, ncolb, beta, st);
}

// emission on cross-section opacities (Sect. 7): each job's Doppler-shifted extinction, then the column
// walk and the hybrid pdf
cudaError_t prep_emission_xsec(int precision, const DevGrid &hg, const XsecDev &xs, const PrepJob *djobs, int njobs,
                               double tau_vert_max, double beta, cudaStream_t st)
{
    cudaError_t e = prep_xsec(precision, hg, xs, djobs, njobs, st);
    if (e != cudaSuccess) return e;
    count_launch(1);
    const bool f64 = precision == GCMC_FP64;
    const int ncolb = emis_col_blocks(hg);
    const dim3 gc((unsigned)ncolb, (unsigned)njobs);
    if (f64) k_emis_column_alpha<double><<<gc, COL_BLOCK, hg.nr * sizeof(double), st>>>(hg, djobs, tau_vert_max);
    else k_emis_column_alpha<float><<<gc, COL_BLOCK, hg.nr * sizeof(float), st>>>(hg, djobs, tau_vert_max);
    return emission_pdf(f64, hg, djobs, njobs, ncolb, beta, st);
}

// ------------------------------------------------------------------ transmission (Doppler cross-sections)
__global__ void k_xsec_cells(DevGrid G, XsecDev xs, int2 *ab, double2 *w, double *fac, float2 *w32, float *dlt)
{
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= G.ncell) return;
    int a, b;
    double wT, wp;
    interp_idx(xs.Tg, xs.nT, (double)G.T[idx], a, wT);
    interp_idx(xs.pg, xs.np, (double)G.p[idx], b, wp);
    ab[idx] = make_int2(a, b);
    w[idx] = make_double2(wT, wp);
    w32[idx] = make_float2((float)wT, (float)wp);
    double v = 0.0;
    if (G.wind) {
        const int i = (int)(idx % G.nlon), j = (int)((idx / G.nlon) % G.nlat), k = (int)(idx / ((int64_t)G.nlon * G.nlat));
        const double lat = 0.5 * (G.lat[j] + G.lat[j + 1]);
        const double th = 0.5 * PI - lat;     // polar angle of the cell
        const double ph = 0.5 * (G.lon[i] + G.lon[i + 1]);
        const double rmid = 0.5 * (G.r[k] + G.r[k + 1]);
        const double u = G.wind[idx], vv = G.wind[G.ncell + idx], ww = G.wind[2 * G.ncell + idx];
        const double dph = ph - xs.view_phi;
        v = u * sin(xs.view_theta) * sin(dph) + (vv * cos(th) - ww * sin(th)) * sin(xs.view_theta) * cos(dph) -
            (vv * sin(th) + ww * cos(th)) * cos(xs.view_theta) +
            xs.omega_rot * rmid * sin(th) * sin(xs.view_theta) * sin(dph);
    }
    fac[idx] = 1.0 - v / C_LIGHT;
    dlt[idx] = (float)(-v / C_LIGHT);   // lambda_eff / lambda_0 - 1, |.| ~ 1e-5: FP32 keeps ~1e-12 absolute
}

// min and max of an FP32 array (one block)
__global__ void k_minmax_f(const float *__restrict__ x, int64_t n, float *out)
{
    __shared__ float smin[32], smax[32];
    float lo = 3.0e38f, hi = -3.0e38f;
    for (int64_t i = threadIdx.x; i < n; i += blockDim.x) {
        lo = fminf(lo, x[i]);
        hi = fmaxf(hi, x[i]);
    }
#pragma unroll
    for (int o = 16; o; o >>= 1) {
        lo = fminf(lo, __shfl_xor_sync(0xffffffffu, lo, o));
        hi = fmaxf(hi, __shfl_xor_sync(0xffffffffu, hi, o));
    }
    if ((threadIdx.x & 31) == 0) {
        smin[threadIdx.x >> 5] = lo;
        smax[threadIdx.x >> 5] = hi;
    }
    __syncthreads();
    if (threadIdx.x == 0) {
        for (int q = 1; q < (int)(blockDim.x >> 5); ++q) {
            lo = fminf(lo, smin[q]);
            hi = fmaxf(hi, smax[q]);
        }
        out[0] = lo;
        out[1] = hi;
    }
}

// FP64 cross-section tables: lambda_eff bracketed and interpolated in FP64
__global__ void k_prep_xsec(DevGrid G, XsecDev xs, const PrepJob *__restrict__ jobs)
{
    const int2 *__restrict__ ab = xs.ab;
    const double2 *__restrict__ w = xs.w;
    const double *__restrict__ fac = xs.fac;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= G.ncell) return;
    const PrepJob pj = jobs[blockIdx.y];
    const double le = pj.lam_m * fac[idx];
    int l;
    const double *lam = xs.lam;
    if (le <= lam[0]) l = -1;
    else if (le >= lam[xs.nl - 1]) l = -2;
    else {
        l = pj.lam_hint;
        if (l < 0) l = 0;
        if (l > xs.nl - 2) l = xs.nl - 2;
        while (lam[l + 1] <= le) ++l;
        while (lam[l] > le) --l;
    }
    const int2 q = ab[idx];
    const int np = xs.np, nTp = xs.nT * xs.np;
    const int o00 = q.x * np + q.y, o10 = (q.x + 1) * np + q.y, o01 = q.x * np + q.y + 1, o11 = (q.x + 1) * np + q.y + 1;
    double wl;
    int l0;
    if (l == -1) { l0 = 0; wl = 0.0; }
    else if (l == -2) { l0 = xs.nl - 2; wl = 1.0; }
    else { l0 = l; wl = (le - lam[l0]) / (lam[l0 + 1] - lam[l0]); }
    const double wT = w[idx].x, wp = w[idx].y;
    double ls[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const double *s = xs.lnsig + (int64_t)(l0 + e) * nTp;
        ls[e] = (1 - wT) * (1 - wp) * s[o00] + wT * (1 - wp) * s[o10] + (1 - wT) * wp * s[o01] + wT * wp * s[o11];
    }
    reinterpret_cast<double *>(pj.rec)[idx] = (double)G.rho[idx] * exp((1.0 - wl) * ls[0] + wl * ls[1]);
}

// FP32 cross-section tables.  The Doppler shift moves lambda_eff by |v_LOS|/c ~ 1e-5 around the job's
// rest wavelength, so the host gives each job the table wavelengths that can bracket any of the grid's
// shifts, as FP32 offsets relative to the rest wavelength (d_l = lambda_l / lambda_0 - 1, from FP64);
// each cell brackets its own shift d (FP32) among them and interpolates in FP32.  Jobs whose window
// reaches a table edge, or needs more than XS_LOCAL wavelengths, bracket lambda_eff in FP64 as the FP64
// kernel does.
__global__ void k_prep_xsec_f32(DevGrid G, XsecDev xs, const PrepJob *__restrict__ jobs)
{
    __shared__ float s_d[XS_LOCAL];
    const PrepJob &pj = jobs[blockIdx.y];
    const int n = pj.xs_n, lo = pj.xs_lo;
    for (int t = threadIdx.x; t < n; t += blockDim.x) s_d[t] = pj.xs_d[t];
    __syncthreads();
    const double *lam = xs.lam;
    const int nl = xs.nl;
    const int64_t idx = (int64_t)blockIdx.x * blockDim.x + threadIdx.x;
    if (idx >= G.ncell) return;
    int l0;
    float wl;
    if (n > 0) {
        const float d = xs.dlt_f[idx];
        int t = 0;
        while (t + 2 < n && s_d[t + 1] <= d) ++t;
        l0 = lo + t;
        wl = __fdividef(d - s_d[t], s_d[t + 1] - s_d[t]);
    } else {
        const double le = pj.lam_m * xs.fac[idx];
        if (le <= lam[0]) {
            l0 = 0;
            wl = 0.0f;
        } else if (le >= lam[nl - 1]) {
            l0 = nl - 2;
            wl = 1.0f;
        } else {
            int l = pj.lam_hint < 0 ? 0 : pj.lam_hint > nl - 2 ? nl - 2 : pj.lam_hint;
            while (lam[l + 1] <= le) ++l;
            while (lam[l] > le) --l;
            l0 = l;
            wl = __fdividef((float)(le - lam[l0]), (float)(lam[l0 + 1] - lam[l0]));
        }
    }
    const int2 q = xs.ab[idx];
    const int np = xs.np, nTp = xs.nT * xs.np;
    const int o00 = q.x * np + q.y, o10 = (q.x + 1) * np + q.y, o01 = q.x * np + q.y + 1, o11 = (q.x + 1) * np + q.y + 1;
    const float2 ww = xs.w32[idx];
    const float wT = ww.x, wp = ww.y;
    float ls[2];
#pragma unroll
    for (int e = 0; e < 2; ++e) {
        const float *sg = xs.lnsig_f + (int64_t)(l0 + e) * nTp;
        ls[e] = (1 - wT) * (1 - wp) * __ldg(sg + o00) + wT * (1 - wp) * __ldg(sg + o10) + (1 - wT) * wp * __ldg(sg + o01) +
                wT * wp * __ldg(sg + o11);
    }
    reinterpret_cast<float *>(pj.rec)[idx] = G.rho[idx] * __expf((1.0f - wl) * ls[0] + wl * ls[1]);
}

cudaError_t xsec_cells(const DevGrid &hg, const XsecDev &xs, int2 *ab, double2 *w, double *fac, float2 *w32, float *dlt,
                       float *minmax, cudaStream_t st)
{
    count_launch(2);
    const unsigned nb = (unsigned)((hg.ncell + PREP_BLOCK - 1) / PREP_BLOCK);
    k_xsec_cells<<<nb, PREP_BLOCK, 0, st>>>(hg, xs, ab, w, fac, w32, dlt);
    k_minmax_f<<<1, 1024, 0, st>>>(dlt, hg.ncell, minmax);
    return cudaGetLastError();
}

cudaError_t prep_xsec(int precision, const DevGrid &hg, const XsecDev &xs, const PrepJob *djobs, int njobs, cudaStream_t st)
{
    count_launch(1);
    const dim3 g1((unsigned)((hg.ncell + PREP_BLOCK - 1) / PREP_BLOCK), (unsigned)njobs);
    if (precision == GCMC_FP64) k_prep_xsec<<<g1, PREP_BLOCK, 0, st>>>(hg, xs, djobs);
    else k_prep_xsec_f32<<<g1, PREP_BLOCK, 0, st>>>(hg, xs, djobs);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ Philox self test
__global__ void k_philox_selftest(const uint32_t *ctr, const uint32_t *key, int n, uint32_t *out_lib, uint32_t *out_cur)
{
    const int t = blockIdx.x * blockDim.x + threadIdx.x;
    if (t >= n) return;
    const uint4 c = make_uint4(ctr[4 * t], ctr[4 * t + 1], ctr[4 * t + 2], ctr[4 * t + 3]);
    const uint2 k = make_uint2(key[2 * t], key[2 * t + 1]);
    const uint4 a = philox10(c, k);
    const uint4 b = curand_Philox4x32_10(c, k);
    out_lib[4 * t] = a.x; out_lib[4 * t + 1] = a.y; out_lib[4 * t + 2] = a.z; out_lib[4 * t + 3] = a.w;
    out_cur[4 * t] = b.x; out_cur[4 * t + 1] = b.y; out_cur[4 * t + 2] = b.z; out_cur[4 * t + 3] = b.w;
}

cudaError_t selftest_philox(const uint32_t *ctr, const uint32_t *key, int n, uint32_t *out_lib, uint32_t *out_cur,
                            cudaStream_t st)
{
    if (n <= 0) return cudaSuccess;
    count_launch(1);
    k_philox_selftest<<<(n + 127) / 128, 128, 0, st>>>(ctr, key, n, out_lib, out_cur);
    return cudaGetLastError();
}

// ------------------------------------------------------------------ random-gather microbenchmark
template <int RB>
__global__ void k_gather(const void *__restrict__ table, uint32_t n, int64_t iters, float *sink)
{
    const uint32_t t = blockIdx.x * blockDim.x + threadIdx.x;
    float acc = 0.0f;
    uint32_t h = t * 0x9E3779B9u + 0x7F4A7C15u;
    for (int64_t it = 0; it < iters; ++it) {
        h ^= h << 13;
        h ^= h >> 17;
        h ^= h << 5;
        const uint32_t idx = __umulhi(h, n);
        if constexpr (RB == 16) {
            const float4 v = __ldg(reinterpret_cast<const float4 *>(table) + idx);
            acc += v.x + v.w;
        } else {
            acc += __ldg(reinterpret_cast<const float *>(table) + idx);
        }
    }
    if (acc == 1.2345f) sink[t] = acc;
}

cudaError_t gather_bench(const void *table, int64_t n_records, int record_bytes, int64_t iters, int blocks, int threads,
                         float *sink, cudaStream_t st)
{
    count_launch(1);
    if (record_bytes == 16) k_gather<16><<<blocks, threads, 0, st>>>(table, (uint32_t)n_records, iters, sink);
    else k_gather<4><<<blocks, threads, 0, st>>>(table, (uint32_t)n_records, iters, sink);
    return cudaGetLastError();
}

}  // namespace gcmc

// ------------------------------------------------------------------ allocation-free emission pdf
// Scratch of gcmc_emission_pdf_noalloc: per-block partial sums and counts (EMIS_SCAN_BLOCK cells per
// block), the job's info block (the pdf kernels write all eight of its slots; only the first three
// are copied out to the caller's totals) and the job record the pdf kernels read.  File-scope device
// memory: one copy per GPU that loads the library, kept until exit.  Every slot read by a kernel is
// written earlier in the same call (partial sums by k_emis_reduce, offsets by k_emis_scan_blocks, the
// info block by k_emis_total and k_emis_scan_blocks, the record by k_noalloc_job), so nothing needs
// clearing between calls; overlapping calls race on it.
namespace {
constexpr int NOALLOC_BLOCKS = GCMC_NOALLOC_MAX_CELLS / gcmc::EMIS_SCAN_BLOCK;
struct __align__(256) NoallocScratch {
    double bsum[NOALLOC_BLOCKS];
    double bcnt[NOALLOC_BLOCKS];
    double info[8];
    gcmc::PrepJob job;
};
static __device__ __align__(256) NoallocScratch g_noalloc;

__global__ void k_noalloc_job(NoallocScratch *sc, double *cdf, double *wcell)
{
    gcmc::PrepJob j;
    memset(&j, 0, sizeof(j));
    j.cdf = reinterpret_cast<long long *>(cdf);
    j.wcell = wcell;
    j.info = sc->info;
    j.bsum = sc->bsum;
    j.bcnt = sc->bcnt;
    sc->job = j;
}

__global__ void k_noalloc_copy(const double *__restrict__ src, double *__restrict__ dst, int64_t n)
{
    for (int64_t i = (int64_t)blockIdx.x * blockDim.x + threadIdx.x; i < n; i += (int64_t)gridDim.x * blockDim.x)
        dst[i] = src[i];
}

// L_tot, the emitting-cell count and the cdf total out of the scratch info block
__global__ void k_noalloc_totals(const NoallocScratch *sc, double *totals)
{
    if (threadIdx.x < 3) totals[threadIdx.x] = sc->info[threadIdx.x];
}

std::atomic<NoallocScratch *> g_noalloc_addr[64];   // per device: address of g_noalloc (host-side lookup)

// byte ranges [a, a + na) and [b, b + nb) share a byte
bool overlaps(const void *a, size_t na, const void *b, size_t nb)
{
    const uintptr_t x = reinterpret_cast<uintptr_t>(a), y = reinterpret_cast<uintptr_t>(b);
    return x < y + nb && y < x + na;
}

// status of the launch just queued (no error was pending when the call began, so one now is its own)
gcmc_status queued_ok()
{
    if (cudaPeekAtLastError() == cudaSuccess) return GCMC_OK;
    cudaGetLastError();
    return GCMC_ERR_CUDA;
}
}  // namespace

extern "C" gcmc_status gcmc_emission_pdf_noalloc(const double *lum, int64_t ncell, double beta, double *cdf,
                                                 double *wcell, double *totals, void *stream)
{
    using namespace gcmc;
    if (!lum || !cdf || !wcell || !totals || ncell < 1 || !(beta >= 0.0 && beta <= 1.0)) return GCMC_ERR_ARG;
    if (ncell > GCMC_NOALLOC_MAX_CELLS) return GCMC_ERR_RANGE;
    const size_t nb = (size_t)ncell * sizeof(double), tb = 3 * sizeof(double);
    // lum may be cdf itself (in place); otherwise no two of the four arrays may share memory
    if ((lum != cdf && overlaps(lum, nb, cdf, nb)) || overlaps(lum, nb, wcell, nb) || overlaps(lum, nb, totals, tb) ||
        overlaps(cdf, nb, wcell, nb) || overlaps(cdf, nb, totals, tb) || overlaps(wcell, nb, totals, tb))
        return GCMC_ERR_ARG;
    // an error left pending by earlier work of the process is not this call's: refuse, and leave it for
    // its owner to read
    if (cudaPeekAtLastError() != cudaSuccess) return GCMC_ERR_CUDA;
    int dev = 0;
    if (cudaGetDevice(&dev) != cudaSuccess || dev < 0 || dev >= 64) return GCMC_ERR_CUDA;
    // set-up once per device, with that device current: the device address of the scratch array
    NoallocScratch *sc = g_noalloc_addr[dev].load();
    if (!sc) {
        void *p = nullptr;
        if (cudaGetSymbolAddress(&p, g_noalloc) != cudaSuccess || !p) {
            cudaGetLastError();
            return GCMC_ERR_CUDA;
        }
        sc = static_cast<NoallocScratch *>(p);
        g_noalloc_addr[dev].store(sc);
    }
    cudaStream_t st = (cudaStream_t)stream;
    const int nblk = (int)((ncell + EMIS_SCAN_BLOCK - 1) / EMIS_SCAN_BLOCK);
    const PrepJob *pj = &sc->job;
    const dim3 g3((unsigned)nblk, 1u);
    gcmc_status s;
    count_launch(1);
    k_noalloc_job<<<1, 1, 0, st>>>(sc, cdf, wcell);
    if ((s = queued_ok()) != GCMC_OK) return s;
    if (lum != cdf) {
        count_launch(1);
        k_noalloc_copy<<<(unsigned)std::min<int64_t>((ncell + 255) / 256, 4096), 256, 0, st>>>(lum, cdf, ncell);
        if ((s = queued_ok()) != GCMC_OK) return s;
    }
    count_launch(1);
    k_emis_reduce<<<g3, EMIS_SCAN_BLOCK, 0, st>>>(ncell, pj);
    if ((s = queued_ok()) != GCMC_OK) return s;
    count_launch(1);
    k_emis_total<<<1, 128, 0, st>>>(nblk, pj, 1, beta);
    if ((s = queued_ok()) != GCMC_OK) return s;
    count_launch(1);
    k_emis_pdf<double><<<g3, EMIS_SCAN_BLOCK, 0, st>>>(ncell, pj, beta);
    if ((s = queued_ok()) != GCMC_OK) return s;
    count_launch(1);
    k_emis_scan_blocks<<<1, 32, 0, st>>>(nblk, pj, 1);
    if ((s = queued_ok()) != GCMC_OK) return s;
    count_launch(1);
    k_emis_cdf_add<double><<<g3, EMIS_SCAN_BLOCK, 0, st>>>(ncell, pj);
    if ((s = queued_ok()) != GCMC_OK) return s;
    count_launch(1);
    k_noalloc_totals<<<1, 32, 0, st>>>(sc, totals);
    return queued_ok();
}
