// Density matrix from Kohn-Sham eigenvectors (gint_density_matrix), Eq. density_matrix:
//   DM_mu,nu(R) = Re Sum_q w_q Sum_n f_n,q c_n,mu,q c*_n,nu,q exp(-i k_q.R).
// Per k point the dense matrix rho(k) = C diag(f) C^H is formed (complex GEMM over the bands,
// planar real / imaginary scratch), then added into every block of the store with its phase
// (the unfolding of gint_unfold, accumulated over k).  FP64 path: CUDA-core complex GEMM with
// 64 x 64 output tiles staged through shared memory (FP64-pipe bound).
//
// TF32x3 path: the complex product is two real GEMMs over K = 2 nbands with the band index and
// the real / imaginary part interleaved (the memory order of C):
//   Re rho = Sum_k A_re[mu][k] B[nu][k],  A_re = C (as reals), B[nu][2n+t] = f_n C[nu][2n+t]
//   Im rho = Sum_k A_im[mu][k] B[nu][k],  A_im[mu][2n] = Im c_mu,n, A_im[mu][2n+1] = -Re c_mu,n
// (the imaginary part is skipped at k = 0, where only Re rho(k) reaches the block store).  The
// band reduction is long (K = 2048 for 1024 bands) and the tensor cores accumulate in FP32 with
// an error that grows with the number of MMA steps, so K is cut into 64-term segments: each
// segment is accumulated in its own TMEM buffer (24 MMA steps, as a 64-point vlocal batch), and
// the epilogue adds the segments with round-to-nearest FP32 additions into a running sum kept in
// TMEM.  The operands are split once per k point into TF32 hi / lo planes (rows padded to 128,
// K to 32, zero-filled); 128 x 128 output tiles, persistent CTAs; 8 producer warps copy the
// planes into the canonical operand layout with cp.async (three stages in flight), one thread
// issues the MMAs, 8 epilogue warps sum the segments.
#include <algorithm>
#include <vector>

#include "gint_device.cuh"
#include "gint_internal.h"
#include "gint_tcgen05.cuh"

using namespace gint;

namespace {

constexpr int kT = 64;      // output tile (rows and columns)
constexpr int kKb = 16;     // bands per shared-memory step
constexpr int kGemmThreads = 256;

// rho(k) = C diag(f) C^H for one k point: C is nbasis x nbands complex (re, im interleaved,
// row-major); out_re / out_im are nbasis x nbasis (planar).  Thread (ty, tx) owns rows
// 4 ty .. 4 ty + 3 and columns tx, tx + 16, tx + 32, tx + 48 of the tile.
__global__ void __launch_bounds__(kGemmThreads)
    k_rhok_f64(const double2 *__restrict__ C, const double *__restrict__ f, int nbasis, int nbands,
               double *__restrict__ out_re, double *__restrict__ out_im)
{
    __shared__ double2 As[kKb][kT + 1];
    __shared__ double2 Bs[kKb][kT + 1];   // f-scaled
    const int tiles = (nbasis + kT - 1) / kT;
    const int tid = threadIdx.x, ty = tid >> 4, tx = tid & 15;
    for (int t = blockIdx.x; t < tiles * tiles; t += gridDim.x) {
        const int m0 = (t / tiles) * kT, n0 = (t % tiles) * kT;
        double re[4][4], im[4][4];
#pragma unroll
        for (int i = 0; i < 4; ++i)
#pragma unroll
            for (int j = 0; j < 4; ++j) re[i][j] = im[i][j] = 0.0;
        for (int b0 = 0; b0 < nbands; b0 += kKb) {
            __syncthreads();
            for (int e = tid; e < kKb * kT; e += kGemmThreads) {
                const int r = e / kKb, b = e - r * kKb;   // consecutive threads: consecutive bands
                const int band = b0 + b;
                double2 a = make_double2(0.0, 0.0), c = make_double2(0.0, 0.0);
                if (band < nbands) {
                    if (m0 + r < nbasis) a = C[(int64_t)(m0 + r) * nbands + band];
                    if (n0 + r < nbasis) {
                        const double2 v = C[(int64_t)(n0 + r) * nbands + band];
                        const double fb = f[band];
                        c = make_double2(fb * v.x, fb * v.y);
                    }
                }
                As[b][r] = a;
                Bs[b][r] = c;
            }
            __syncthreads();
#pragma unroll 4
            for (int b = 0; b < kKb; ++b) {
                double2 a[4], c[4];
#pragma unroll
                for (int i = 0; i < 4; ++i) a[i] = As[b][4 * ty + i];
#pragma unroll
                for (int j = 0; j < 4; ++j) c[j] = Bs[b][tx + 16 * j];
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        // a c* = (ar cr + ai ci) + i (ai cr - ar ci)
                        re[i][j] = fma(a[i].x, c[j].x, fma(a[i].y, c[j].y, re[i][j]));
                        im[i][j] = fma(a[i].y, c[j].x, fma(-a[i].x, c[j].y, im[i][j]));
                    }
            }
        }
#pragma unroll
        for (int i = 0; i < 4; ++i) {
            const int r = m0 + 4 * ty + i;
            if (r >= nbasis) continue;
#pragma unroll
            for (int j = 0; j < 4; ++j) {
                const int c = n0 + tx + 16 * j;
                if (c < nbasis) {
                    out_re[(int64_t)r * nbasis + c] = re[i][j];
                    out_im[(int64_t)r * nbasis + c] = im[i][j];
                }
            }
        }
    }
}

// DM(block b) (+)= w Re[rho(k) exp(-i 2 pi kappa.n_b)] for every block; one CTA per block
__global__ void k_unfold_acc(const int *__restrict__ keys, int64_t nblocks, const int *__restrict__ orboff,
                             const int64_t *__restrict__ off, const double *__restrict__ re,
                             const double *__restrict__ im, double k1, double k2, double k3, double w, int nbasis,
                             int first, int use_im, double *__restrict__ X)
{
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int *k = keys + 5 * b;
        const int I = k[0], J = k[1];
        const int r0 = orboff[I], nI = orboff[I + 1] - r0;
        const int c0 = orboff[J], nJ = orboff[J + 1] - c0;
        double s, c;
        sincospi(2.0 * (k1 * k[2] + k2 * k[3] + k3 * k[4]), &s, &c);
        for (int e = threadIdx.x; e < nI * nJ; e += blockDim.x) {
            const int mu = e / nJ, nu = e - mu * nJ;
            const int64_t g = (int64_t)(r0 + mu) * nbasis + (c0 + nu);
            const double v = w * (use_im ? fma(re[g], c, im[g] * s) : re[g] * c);   // Re[(re + i im)(c - i s)]
            X[off[b] + e] = first ? v : X[off[b] + e] + v;
        }
    }
}

// ------------------------------------------------------------------ tensor-core path
constexpr int kDmProd = 256;                 // producer threads (warps 0-7)
constexpr int kDmEpi0 = 256;                 // epilogue warps 8-15 (TMEM lane quadrant = warp % 4)
constexpr int kDmMma = 512;                  // MMA-issue thread (warp 16)
constexpr int kDmThreads = 544;
constexpr int kDmBM = 128, kDmBN = 128;      // output tile
constexpr int kDmKC = 32;                    // K values per chunk (TF32x3W: 8 core matrices of 4)
constexpr int kDmSeg = 64;                   // K values per TMEM segment
constexpr int kDmStages = 3;
constexpr int kDmSumCol = 256;               // TMEM column of the running sum

struct DmSmem {
    static constexpr int ARR = arr_bytes<TF32x3W>(128);                    // one operand term
    static constexpr int STAGE = 4 * ARR;                                    // A hi, lo, B hi, lo
    static constexpr int OFF_BAR = kDmStages * STAGE;                        // 16 mbarriers
    static constexpr int OFF_MISC = OFF_BAR + 16 * 8;
    static constexpr int TOTAL = OFF_MISC + 64;
};

// TF32 hi / lo planes of the three operands, each [Np][Kp] floats (Np = nbasis rounded up to 128,
// Kp = 2 nbands rounded up to 32, zero-filled): plane 2p + t holds term t of operand p, with
// p = 0: A_re (C as reals), 1: A_im (pairs (Im c, -Re c)), 2: B (f_n C as reals).
__global__ void k_dm_split(const double *__restrict__ C, const double *__restrict__ f, int nbasis, int nbands,
                           int Np, int Kp, int with_im, float *__restrict__ planes)
{
    const int K = 2 * nbands;
    const int64_t plane = (int64_t)Np * Kp;
    const int64_t n = plane;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int row = (int)(e / Kp), k = (int)(e - (int64_t)row * Kp);
        double a = 0.0, ai = 0.0, b = 0.0;
        if (row < nbasis && k < K) {
            const double v = C[(int64_t)row * K + k];
            const double w = C[(int64_t)row * K + (k ^ 1)];   // the other part of the same number
            a = v;
            ai = (k & 1) ? -w : w;                             // (Im c, -Re c)
            b = f[k >> 1] * v;
        }
        const double vals[3] = {a, ai, b};
#pragma unroll
        for (int p = 0; p < 3; ++p) {
            if (p == 1 && !with_im) continue;
            const float x = (float)vals[p];
            const float hi = tf32_rna(x);
            planes[(2 * p) * plane + e] = hi;
            planes[(2 * p + 1) * plane + e] = tf32_rna(x - hi);
        }
    }
}

// rho(k) part (0: real, 1: imaginary) of C diag(f) C^H into out (nbasis x nbasis, row-major)
__global__ void __launch_bounds__(kDmThreads, 1)
    k_rhok_tc(Plan P, const float *__restrict__ planes, int Np, int Kp, int nbasis, int part, double *__restrict__ out)
{
    using S = TF32x3W;
    using L = DmSmem;
    constexpr int SBO = S::KCM * kLBO;
    extern __shared__ __align__(1024) unsigned char sm[];
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::OFF_BAR);
    uint64_t *full = bars, *empty = bars + kDmStages, *segfull = bars + 2 * kDmStages;
    uint64_t *segempty = segfull + 2, *fin = segfull + 4;
    static_assert(2 * kDmStages + 5 <= 16, "mbarrier space");
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(sm + L::OFF_MISC);
    volatile int *pflag = reinterpret_cast<volatile int *>(sm + L::OFF_MISC + 4);
    volatile int *eflag = reinterpret_cast<volatile int *>(sm + L::OFF_MISC + 8);
    const int tid = threadIdx.x, warp = tid >> 5;
    if (tid == 0) {
        for (int i = 0; i < kDmStages; ++i) {
            mbar_init(&full[i], 1);
            mbar_init(&empty[i], 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(&segfull[i], 1);
            mbar_init(&segempty[i], 256);
        }
        mbar_init(fin, 1);
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(su32(tmem_base)),
                     "r"(kTmemCols));
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_base;
    const int nt = Np / kDmBM;
    const int ntiles = nt * nt;
    const int nchunk = Kp / kDmKC;
    const int nseg = (Kp + kDmSeg - 1) / kDmSeg;
    const int64_t plane = (int64_t)Np * Kp;
    constexpr int CPS = kDmSeg / kDmKC;     // chunks per segment

    if (tid < kDmProd) {
        // ------------------------------------------------------------ producers
        // chunk g is copied into stage g % 3 with cp.async; its completion is awaited one
        // chunk later (so two chunks are in flight), then fenced for the async proxy and
        // announced on full[stage]
        const int pt = tid;
        int g = 0;
        bool ok = true;
        const float *Ah = planes + (2 * part) * plane, *Al = Ah + plane;
        const float *Bh = planes + 4 * plane, *Bl = Bh + plane;
        auto announce = [&](int gg) {
            cp_async_wait_group1();
            fence_async_smem();
            named_sync(1, kDmProd);
            if (pt == 0) mbar_arrive(&full[gg % kDmStages]);
        };
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int m0 = (t / nt) * kDmBM, n0 = (t % nt) * kDmBN;
            for (int ch = 0; ch < nchunk && ok; ++ch, ++g) {
                const int stage = g % kDmStages;
                if (g >= kDmStages)
                    ok = role_wait(&empty[stage], ((g / kDmStages) - 1) & 1, P, pt, pflag, 1, kDmProd);
                if (!ok) break;
                unsigned char *base = sm + stage * L::STAGE;
                const int k0 = ch * kDmKC;
                // 128 A rows and 128 B rows x 8 core-matrix columns x 2 terms, 16 bytes each
                for (int w = pt; w < 4 * 128 * S::KCM; w += kDmProd) {
                    const int term = w / (2 * 128 * S::KCM);
                    const int ww = w - term * (2 * 128 * S::KCM);
                    const int isb = ww >= 128 * S::KCM;
                    const int w2 = isb ? ww - 128 * S::KCM : ww;
                    const int kc = w2 % S::KCM, row = w2 / S::KCM;
                    const float *src = (isb ? (term ? Bl : Bh) : (term ? Al : Ah)) +
                                       (int64_t)((isb ? n0 : m0) + row) * Kp + k0 + kc * S::CG;
                    cp_async16(base + (isb ? 2 : 0) * L::ARR + term * L::ARR + cm_off<S>(row, kc), src);
                }
                cp_async_commit();
                if (g > 0) announce(g - 1);   // the previous chunk has landed
            }
        }
        if (ok && g > 0) {
            cp_async_wait_all();
            fence_async_smem();
            named_sync(1, kDmProd);
            if (pt == 0) mbar_arrive(&full[(g - 1) % kDmStages]);
        }
        cp_async_wait_all();
    } else if (tid >= kDmMma) {
        // ------------------------------------------------------------ MMA issue (one thread)
        if (tid == kDmMma) {
            int g = 0, u = 0;   // chunk and segment counters
            bool ok = true;
            const uint32_t id = idesc<S>(kDmBM, kDmBN);
            for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
                for (int ch = 0; ch < nchunk && ok; ++ch, ++g) {
                    const int stage = g % kDmStages;
                    const bool seg0 = ch % CPS == 0, seg1 = ch % CPS == CPS - 1 || ch == nchunk - 1;
                    const int sb = u & 1;
                    ok = !aborted(P) && mbar_wait(&full[stage], (g / kDmStages) & 1, P.spin_limit);
                    if (ok && seg0 && u >= 2)   // the epilogue has taken segment u - 2 out of buffer sb
                        ok = !aborted(P) && mbar_wait(&segempty[sb], ((u >> 1) - 1) & 1, P.spin_limit);
                    if (!ok) {
                        report_timeout(P);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = su32(sm + stage * L::STAGE), b0 = a0 + 2 * L::ARR;
#pragma unroll
                    for (int ks = 0; ks < S::KCM / 2; ++ks)
#pragma unroll
                        for (int q = 0; q < S::NPROD; ++q) {
                            const uint64_t da = sdesc(a0 + term(S::PA, q) * L::ARR + ks * 2 * kLBO, SBO);
                            const uint64_t db = sdesc(b0 + term(S::PB, q) * L::ARR + ks * 2 * kLBO, SBO);
                            const uint32_t acc = (seg0 && ks == 0 && q == 0) ? 0u : 1u;
                            umma<false>(tmem + sb * kDmBN, da, db, id, acc);
                        }
                    umma_commit(&empty[stage]);
                    if (seg1) {
                        umma_commit(&segfull[sb]);
                        ++u;
                    }
                }
            }
            umma_commit(fin);
            if (!mbar_wait(fin, 0, kDrainBudget)) report_timeout(P);
        }
    } else {
        // ------------------------------------------------------------ epilogue: segment sums
        const int et = tid - kDmEpi0, ew = et >> 5, lane = et & 31;
        const int q = ew & 3, hh = ew >> 2;   // TMEM lane quadrant, column half
        const int row = q * 32 + lane;
        int u = 0;
        bool ok = true;
        for (int t = blockIdx.x; t < ntiles && ok; t += gridDim.x) {
            const int m0 = (t / nt) * kDmBM, n0 = (t % nt) * kDmBN;
            for (int sg = 0; sg < nseg; ++sg, ++u) {
                const int sb = u & 1;
                if (!role_wait(&segfull[sb], (u >> 1) & 1, P, et, eflag, 2, 256)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t lrow = (uint32_t)(q * 32) << 16;
#pragma unroll 1
                for (int c = 0; c < 4; ++c) {
                    const int col = hh * 64 + c * 16;
                    float v[16], acc[16];
                    tmem_ld16(tmem + lrow + (uint32_t)(sb * kDmBN + col), v);
                    if (sg > 0) {
                        tmem_ld16(tmem + lrow + (uint32_t)(kDmSumCol + col), acc);
#pragma unroll
                        for (int j = 0; j < 16; ++j) acc[j] += v[j];
                    } else {
#pragma unroll
                        for (int j = 0; j < 16; ++j) acc[j] = v[j];
                    }
                    if (sg + 1 < nseg) {
                        tmem_st16(tmem + lrow + (uint32_t)(kDmSumCol + col), acc);
                    } else if (m0 + row < nbasis) {
                        double *o = out + (int64_t)(m0 + row) * nbasis + n0 + col;
#pragma unroll
                        for (int j = 0; j < 16; ++j)
                            if (n0 + col + j < nbasis) o[j] = f2d(acc[j]);
                    }
                }
                tc_fence_before();
                mbar_arrive(&segempty[sb]);
                // the running sum is read again by this thread only (wait::st above orders it);
                // the barrier of the next role_wait separates the flag reads
                named_sync(2, 256);
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

gint_status check(gint_handle h, const char *who)
{
    if (!h) {
        set_error("%s: null handle", who);
        return GINT_EINVAL;
    }
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, who);
    if (dev != h->device) {
        set_error("%s: current device %d differs from the handle's device %d", who, dev, h->device);
        return GINT_EINVAL;
    }
    return GINT_OK;
}

}  // namespace

namespace gint {
gint_status ensure_kspace_tables(gint_handle h);
}

extern "C" gint_status gint_density_matrix(gint_handle h, int nk, const double *kfrac, const double *w, int nbands,
                                           const double *C_dev, const double *f_dev, double *DM_dev, gint_prec prec,
                                           void *stream)
{
    gint_status st = check(h, "gint_density_matrix");
    if (st != GINT_OK) return st;
    if (!kfrac || !w || !C_dev || !f_dev || !DM_dev || nk < 1 || nbands < 1 ||
        (prec != GINT_FP64 && prec != GINT_TF32X3)) {
        set_error("gint_density_matrix: null buffer, nk < 1, nbands < 1 or a precision other than FP64, TF32X3");
        return GINT_EINVAL;
    }
    if ((st = ensure_kspace_tables(h)) != GINT_OK) return st;
    cudaStream_t s = (cudaStream_t)stream;
    const int64_t N = h->info.nbasis;
    cudaError_t e;
    const size_t need = sizeof(double) * 2 * N * N;
    if (h->dm_scratch_bytes < need) {
        if (h->d_dm_scratch) cudaFree(h->d_dm_scratch);
        h->d_dm_scratch = nullptr;
        h->dm_scratch_bytes = 0;
        if ((e = cudaMalloc((void **)&h->d_dm_scratch, need)) != cudaSuccess)
            return cuda_fail(e, "gint_density_matrix: allocate");
        h->dm_scratch_bytes = need;
    }
    const int Np = (int)((N + kDmBM - 1) / kDmBM) * kDmBM, Kp = (2 * nbands + kDmKC - 1) / kDmKC * kDmKC;
    const size_t need_planes = prec == GINT_TF32X3 ? sizeof(float) * 6 * (size_t)Np * Kp : 0;
    if (h->dm_planes_bytes < need_planes) {
        if (h->d_dm_planes) cudaFree(h->d_dm_planes);
        h->d_dm_planes = nullptr;
        h->dm_planes_bytes = 0;
        if ((e = cudaMalloc((void **)&h->d_dm_planes, need_planes)) != cudaSuccess)
            return cuda_fail(e, "gint_density_matrix: allocate");
        h->dm_planes_bytes = need_planes;
    }
    double *re = h->d_dm_scratch, *im = re + N * N;
    const int tiles = (int)((N + kT - 1) / kT);
    const int grid = std::min(tiles * tiles, 8 * h->nsm);
    const int tiles_tc = (int)((N + kDmBM - 1) / kDmBM);
    if (prec == GINT_TF32X3 &&
        (e = cudaFuncSetAttribute(k_rhok_tc, cudaFuncAttributeMaxDynamicSharedMemorySize, DmSmem::TOTAL)) != cudaSuccess)
        return cuda_fail(e, "gint_density_matrix: attribute");
    for (int q = 0; q < nk; ++q) {
        const double2 *Cq = (const double2 *)C_dev + (int64_t)q * N * nbands;
        const double *fq = f_dev + (int64_t)q * nbands;
        // at k = 0 only Re rho(k) reaches the block store
        const bool use_im = kfrac[3 * q] != 0.0 || kfrac[3 * q + 1] != 0.0 || kfrac[3 * q + 2] != 0.0;
        if (prec == GINT_FP64) {
            k_rhok_f64<<<grid, kGemmThreads, 0, s>>>(Cq, fq, (int)N, nbands, re, im);
        } else {
            const int g3 = std::min(tiles_tc * tiles_tc, h->nsm);
            const int64_t n = (int64_t)Np * Kp;
            k_dm_split<<<(int)std::min<int64_t>((n + 255) / 256, 8 * h->nsm), 256, 0, s>>>(
                (const double *)Cq, fq, (int)N, nbands, Np, Kp, use_im, h->d_dm_planes);
            for (int part = 0; part < (use_im ? 2 : 1); ++part)
                k_rhok_tc<<<g3, kDmThreads, DmSmem::TOTAL, s>>>(h->plan, h->d_dm_planes, Np, Kp, (int)N, part,
                                                                 part == 0 ? re : im);
        }
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gint_density_matrix: rho(k)");
        if (h->info.nblocks > 0) {
            const int g2 = (int)std::min<int64_t>(h->info.nblocks, 16 * h->nsm);
            k_unfold_acc<<<g2, 256, 0, s>>>(h->ks.d_keys, h->info.nblocks, h->ks.d_orboff, (const int64_t *)h->d_blkoff,
                                            re, im, kfrac[3 * q], kfrac[3 * q + 1], kfrac[3 * q + 2], w[q], (int)N,
                                            q == 0, prec == GINT_FP64 || use_im, DM_dev);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gint_density_matrix: unfold");
        }
    }
    h->last_stream = s;
    return GINT_OK;
}
