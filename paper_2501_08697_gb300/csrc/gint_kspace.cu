// k-space transforms of the block store (gint_fold / gint_unfold).
//
// Folding (Sec. IV.B): X_mu,nu(k) = Sum_R X_mu,nu(R) exp(i k.R), R over all valid
// neighbouring cells, into dense nbasis x nbasis complex matrices; unfolding (Eq.
// density_matrix): X_mu,nu(R) = Re Sum_k w_k X_mu,nu(k) exp(-i k.R).  Both are memory-bound:
// the dense matrices (16 bytes per entry and k point) dominate the traffic.  Blocks with the
// same atom pair (I, J) are consecutive in the store (keys sorted by I, J, n), so folding runs
// over all atom pairs, one CTA at a time per pair: every entry of the pair's dense sub-block is
// summed over the pair's R in registers and written exactly once (zeros for pairs without a
// block), without atomics or a separate clearing pass.  Phases exp(i 2 pi kappa.n) are
// tabulated once per call (FP64 sincospi) and read by all threads of a block.
#include <algorithm>
#include <vector>

#include "gint_internal.h"

using namespace gint;

namespace {

constexpr int kMaxK = 4096;
constexpr int kFoldThreads = 256;
constexpr int kKq = 4;   // k points per register pass of the fold kernel

__global__ void k_phase(const int *__restrict__ keys, int64_t nblocks, const double *__restrict__ kv, int nk,
                        double2 *__restrict__ phase)
{
    const int64_t n = nblocks * nk;
    for (int64_t e = blockIdx.x * (int64_t)blockDim.x + threadIdx.x; e < n; e += (int64_t)gridDim.x * blockDim.x) {
        const int64_t b = e / nk;
        const int q = (int)(e - b * nk);
        const int *k = keys + 5 * b;
        const double t = kv[4 * q] * k[2] + kv[4 * q + 1] * k[3] + kv[4 * q + 2] * k[4];   // turns
        double s, c;
        sincospi(2.0 * t, &s, &c);
        phase[e] = make_double2(c, s);
    }
}

// One CTA per dense row (orbital mu of atom I) for every k point, so each warp writes
// consecutive entries of one row.  Column c belongs to atom J = col_atom[c]; the pair's
// blocks (one per R) are summed in registers, k points kKq at a time.
__global__ void __launch_bounds__(kFoldThreads)
    k_fold(const int *__restrict__ pair, const int *__restrict__ grp, const int *__restrict__ col_atom, int natoms,
           const int *__restrict__ orboff, const int64_t *__restrict__ off, const double *__restrict__ X,
           const double2 *__restrict__ phase, int nk, int64_t nbasis, double2 *__restrict__ Xk)
{
    for (int r = blockIdx.x; r < nbasis; r += gridDim.x) {
        const int I = col_atom[r], mu = r - orboff[I];
        for (int c = threadIdx.x; c < nbasis; c += blockDim.x) {
            const int J = col_atom[c];
            const int c0 = orboff[J], nJ = orboff[J + 1] - c0, nu = c - c0;
            const int gi = pair[I * natoms + J];
            const int b0 = gi >= 0 ? grp[gi] : 0, b1 = gi >= 0 ? grp[gi + 1] : 0;
            double2 *out = Xk + (int64_t)r * nbasis + c;
            for (int q0 = 0; q0 < nk; q0 += kKq) {
                double re[kKq], im[kKq];
#pragma unroll
                for (int j = 0; j < kKq; ++j) re[j] = im[j] = 0.0;
                for (int b = b0; b < b1; ++b) {
                    const double x = X[off[b] + mu * nJ + nu];
                    const double2 *ph = phase + (int64_t)b * nk + q0;
#pragma unroll
                    for (int j = 0; j < kKq; ++j)
                        if (q0 + j < nk) {
                            const double2 p = ph[j];
                            re[j] = fma(x, p.x, re[j]);
                            im[j] = fma(x, p.y, im[j]);
                        }
                }
#pragma unroll
                for (int j = 0; j < kKq; ++j)
                    if (q0 + j < nk) out[(int64_t)(q0 + j) * nbasis * nbasis] = make_double2(re[j], im[j]);
            }
        }
    }
}

// One CTA per block: its entries are read from the dense matrices (the sub-blocks of one atom
// pair stay in L1/L2 across the pair's R) and summed over the k points.
__global__ void __launch_bounds__(kFoldThreads)
    k_unfold(const int *__restrict__ keys, int64_t nblocks, const int *__restrict__ orboff,
             const int64_t *__restrict__ off, const double2 *__restrict__ Xk, const double2 *__restrict__ phase,
             const double *__restrict__ kv, int nk, int64_t nbasis, double *__restrict__ X)
{
    for (int64_t b = blockIdx.x; b < nblocks; b += gridDim.x) {
        const int I = keys[5 * b], J = keys[5 * b + 1];
        const int r0 = orboff[I], nI = orboff[I + 1] - r0;
        const int c0 = orboff[J], nJ = orboff[J + 1] - c0;
        for (int e = threadIdx.x; e < nI * nJ; e += blockDim.x) {
            const int mu = e / nJ, nu = e - mu * nJ;
            const double2 *in = Xk + (int64_t)(r0 + mu) * nbasis + (c0 + nu);
            double acc = 0.0;
            for (int q = 0; q < nk; ++q) {
                const double2 z = in[(int64_t)q * nbasis * nbasis];
                const double2 p = phase[b * nk + q];
                // Re[z exp(-i theta)] = re cos + im sin
                acc = fma(kv[4 * q + 3], fma(z.x, p.x, z.y * p.y), acc);
            }
            X[off[b] + e] = acc;
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
// device tables of the block keys, (I, J) groups and orbital offsets (once per handle)
gint_status ensure_kspace_tables(gint_handle h)
{
    auto &K = h->ks;
    if (K.d_keys) return GINT_OK;
    const int64_t nb = h->info.nblocks;
    std::vector<int> grp{0};
    for (int64_t b = 1; b < nb; ++b)
        if (h->keys[5 * b] != h->keys[5 * (b - 1)] || h->keys[5 * b + 1] != h->keys[5 * (b - 1) + 1])
            grp.push_back((int)b);
    grp.push_back((int)nb);
    if (nb == 0) grp.assign(1, 0);
    std::vector<int> oo(h->natoms + 1, 0);
    for (int I = 0; I < h->natoms; ++I) oo[I + 1] = oo[I] + h->norb_atom[I];
    std::vector<int> colatom(std::max(1, oo[h->natoms]));
    for (int I = 0; I < h->natoms; ++I)
        for (int o = oo[I]; o < oo[I + 1]; ++o) colatom[o] = I;
    std::vector<int> pair((size_t)h->natoms * h->natoms, -1);
    for (size_t g = 0; g + 1 < grp.size(); ++g) {
        const int b = grp[g], I = h->keys[5 * b], J = h->keys[5 * b + 1];
        pair[(size_t)I * h->natoms + J] = (int)g;
    }
    cudaError_t e;
    if ((e = cudaMalloc((void **)&K.d_keys, sizeof(int) * std::max<int64_t>(1, 5 * nb))) != cudaSuccess ||
        (e = cudaMalloc((void **)&K.d_grp, sizeof(int) * grp.size())) != cudaSuccess ||
        (e = cudaMalloc((void **)&K.d_pair, sizeof(int) * pair.size())) != cudaSuccess ||
        (e = cudaMalloc((void **)&K.d_colatom, sizeof(int) * colatom.size())) != cudaSuccess ||
        (e = cudaMalloc((void **)&K.d_orboff, sizeof(int) * oo.size())) != cudaSuccess)
        return cuda_fail(e, "gint_fold: allocate tables");
    if ((nb > 0 && (e = cudaMemcpy(K.d_keys, h->keys.data(), sizeof(int) * 5 * nb, cudaMemcpyHostToDevice)) != cudaSuccess) ||
        (e = cudaMemcpy(K.d_grp, grp.data(), sizeof(int) * grp.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(K.d_pair, pair.data(), sizeof(int) * pair.size(), cudaMemcpyHostToDevice)) != cudaSuccess ||
        (e = cudaMemcpy(K.d_colatom, colatom.data(), sizeof(int) * colatom.size(), cudaMemcpyHostToDevice)) !=
            cudaSuccess ||
        (e = cudaMemcpy(K.d_orboff, oo.data(), sizeof(int) * oo.size(), cudaMemcpyHostToDevice)) != cudaSuccess)
        return cuda_fail(e, "gint_fold: upload tables");
    K.ngroups = (int)grp.size() - 1;
    return GINT_OK;
}

}  // namespace gint

namespace {

// k points (and weights) on the device and the phase table of every block, on stream s
gint_status prepare_k(gint_handle h, int nk, const double *kfrac, const double *w, cudaStream_t s, const char *who)
{
    auto &K = h->ks;
    cudaError_t e;
    if (nk > K.cap) {
        if (K.d_kvec) cudaFree(K.d_kvec);
        if (K.d_phase) cudaFree(K.d_phase);
        K.d_kvec = nullptr;
        K.d_phase = nullptr;
        K.cap = 0;
        if ((e = cudaMalloc((void **)&K.d_kvec, sizeof(double) * 4 * nk)) != cudaSuccess ||
            (e = cudaMalloc((void **)&K.d_phase, sizeof(double2) * std::max<int64_t>(1, h->info.nblocks) * nk)) !=
                cudaSuccess)
            return cuda_fail(e, who);
        K.cap = nk;
    }
    std::vector<double> kv(4 * nk);
    for (int q = 0; q < nk; ++q) {
        for (int c = 0; c < 3; ++c) kv[4 * q + c] = kfrac[3 * q + c];
        kv[4 * q + 3] = w ? w[q] : 0.0;
    }
    // from pageable memory: cudaMemcpyAsync returns once kv has been staged for the transfer,
    // so kv may go out of scope
    if ((e = cudaMemcpyAsync(K.d_kvec, kv.data(), sizeof(double) * 4 * nk, cudaMemcpyHostToDevice, s)) != cudaSuccess)
        return cuda_fail(e, who);
    const int64_t n = h->info.nblocks * nk;
    if (n > 0) {
        const int grid = (int)std::min<int64_t>((n + 255) / 256, 4 * h->nsm);
        k_phase<<<grid, 256, 0, s>>>(K.d_keys, h->info.nblocks, K.d_kvec, nk, (double2 *)K.d_phase);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, who);
    }
    return GINT_OK;
}

}  // namespace

extern "C" gint_status gint_fold(gint_handle h, const double *X_dev, int nk, const double *kfrac, double *Xk_dev,
                                 void *stream)
{
    gint_status st = check(h, "gint_fold");
    if (st != GINT_OK) return st;
    if (!X_dev || !kfrac || !Xk_dev || nk < 1 || nk > kMaxK) {
        set_error("gint_fold: null buffer or nk outside 1..%d", kMaxK);
        return GINT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_kspace_tables(h)) != GINT_OK || (st = prepare_k(h, nk, kfrac, nullptr, s, "gint_fold")) != GINT_OK)
        return st;
    const int64_t N = h->info.nbasis;
    const int grid = (int)std::min<int64_t>(N, 32 * h->nsm);
    k_fold<<<grid, kFoldThreads, 0, s>>>(h->ks.d_pair, h->ks.d_grp, h->ks.d_colatom, h->natoms, h->ks.d_orboff,
                                         (const int64_t *)h->d_blkoff, X_dev, (const double2 *)h->ks.d_phase, nk, N,
                                         (double2 *)Xk_dev);
    cudaError_t e = cudaGetLastError();
    if (e != cudaSuccess) return cuda_fail(e, "gint_fold: launch");
    h->last_stream = s;
    return GINT_OK;
}

extern "C" gint_status gint_unfold(gint_handle h, const double *Xk_dev, int nk, const double *kfrac, const double *w,
                                   double *X_dev, void *stream)
{
    gint_status st = check(h, "gint_unfold");
    if (st != GINT_OK) return st;
    if (!X_dev || !kfrac || !w || !Xk_dev || nk < 1 || nk > kMaxK) {
        set_error("gint_unfold: null buffer or nk outside 1..%d", kMaxK);
        return GINT_EINVAL;
    }
    cudaStream_t s = (cudaStream_t)stream;
    if ((st = ensure_kspace_tables(h)) != GINT_OK || (st = prepare_k(h, nk, kfrac, w, s, "gint_unfold")) != GINT_OK)
        return st;
    cudaError_t e;
    if (h->info.nblocks > 0) {
        const int grid = (int)std::min<int64_t>(h->info.nblocks, 16 * h->nsm);
        k_unfold<<<grid, kFoldThreads, 0, s>>>(h->ks.d_keys, h->info.nblocks, h->ks.d_orboff,
                                               (const int64_t *)h->d_blkoff, (const double2 *)Xk_dev,
                                               (const double2 *)h->ks.d_phase, h->ks.d_kvec, nk, h->info.nbasis, X_dev);
        if ((e = cudaGetLastError()) != cudaSuccess) return cuda_fail(e, "gint_unfold: launch");
    }
    h->last_stream = s;
    return GINT_OK;
}
