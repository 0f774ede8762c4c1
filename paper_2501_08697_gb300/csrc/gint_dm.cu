// Density matrix from Kohn-Sham eigenvectors (gint_density_matrix), Eq. density_matrix:
//   DM_mu,nu(R) = Re Sum_q w_q Sum_n f_n,q c_n,mu,q c*_n,nu,q exp(-i k_q.R).
// Per k point the dense matrix rho(k) = C diag(f) C^H is formed (complex GEMM over the bands,
// planar real / imaginary scratch), then added into every block of the store with its phase
// (the unfolding of gint_unfold, accumulated over k).  FP64 path: CUDA-core complex GEMM with
// 64 x 64 output tiles staged through shared memory (FP64-pipe bound).
#include <algorithm>
#include <vector>

#include "gint_internal.h"

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
                             int first, double *__restrict__ X)
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
            const double v = w * fma(re[g], c, im[g] * s);   // Re[(re + i im)(c - i s)]
            X[off[b] + e] = first ? v : X[off[b] + e] + v;
        }
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
    if (!kfrac || !w || !C_dev || !f_dev || !DM_dev || nk < 1 || nbands < 1 || prec != GINT_FP64) {
        set_error("gint_density_matrix: null buffer, nk < 1, nbands < 1 or a precision other than FP64");
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
    double *re = h->d_dm_scratch, *im = re + N * N;
    const int tiles = (int)((N + kT - 1) / kT);
    const int grid = std::min(tiles * tiles, 8 * h->nsm);
    for (int q = 0; q < nk; ++q) {
        const double2 *Cq = (const double2 *)C_dev + (int64_t)q * N * nbands;
        k_rhok_f64<<<grid, kGemmThreads, 0, s>>>(Cq, f_dev + (int64_t)q * nbands, (int)N, nbands, re, im);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gint_density_matrix: rho(k)");
        if (h->info.nblocks > 0) {
            const int g2 = (int)std::min<int64_t>(h->info.nblocks, 16 * h->nsm);
            k_unfold_acc<<<g2, 256, 0, s>>>(h->ks.d_keys, h->info.nblocks, h->ks.d_orboff, (const int64_t *)h->d_blkoff,
                                            re, im, kfrac[3 * q], kfrac[3 * q + 1], kfrac[3 * q + 2], w[q], (int)N,
                                            q == 0, DM_dev);
            if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gint_density_matrix: unfold");
        }
    }
    h->last_stream = s;
    return GINT_OK;
}
