// CUDA-core (FMA) kernels of libgint: the FP64 and FP32 grid integrations.
//
// vlocal (Sec. IV.B grid integral of the local potential): per grid batch, the orbital
// values Phi[p][mu] of every atom image that reaches the batch are evaluated into shared
// memory; the batch contraction P = Phi^T diag(V) Phi dV is formed tile by tile (only the
// upper triangle of 32 x 32 tiles, P is symmetric) and added into the block store in FP64.
// Each unordered orbital pair is added once, into the canonical member of its partner pair
// {(I,J,R), (J,I,-R)}; a mirror kernel fills the other member afterwards.
//
// rho/force (Eq. density_matrix and the Pulay term of Eq. force_lcao): per batch,
// Psi = Phi D_b with D_b gathered from the block store, rho(p) = Sum_mu Phi[p][mu] Psi[p][mu],
// and F_I += 2 dV Sum_p V(p) Sum_{mu in I} grad phi_mu(p) Psi[p][mu] (D block-symmetric).
#include <cstdio>

#include "gint_device.cuh"

namespace gint {

namespace {

constexpr int kThreads = 256;
constexpr int kSubPts = 64;     // points per shared-memory sub-batch (vlocal)
constexpr int kRhoPts = 128;    // most points per sub-batch (rho/force)
constexpr int kDChunk = 16;     // rows of D staged at a time (rho/force)
constexpr int kRhoTile = 8192;  // elements of the Phi / Psi tile (points x padded orbitals)
constexpr int kDRegs = kDChunk * kMaxNb / kThreads;   // staged D values per thread

struct SlotSh {
    int atom, species, orb_off, norb;
    double d0[3];
};

__device__ __forceinline__ void unpack_dims(int dims, int &n1, int &n2, int &n3)
{
    n1 = dims & 255;
    n2 = (dims >> 8) & 255;
    n3 = (dims >> 16) & 255;
}

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) k_vlocal_simt(Plan P, const double *__restrict__ V, double *H)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SlotSh *sl = reinterpret_cast<SlotSh *>(smem);                                   // kMaxSlots
    int *tbl = reinterpret_cast<int *>(sl + kMaxSlots);                              // kMaxSlots^2
    unsigned char *oslot = reinterpret_cast<unsigned char *>(tbl + kMaxSlots * kMaxSlots);  // kMaxNb
    unsigned char *oidx = oslot + kMaxNb;                                             // kMaxNb
    T *Vs = reinterpret_cast<T *>(oidx + kMaxNb);                                     // kSubPts
    T *Phi = Vs + kSubPts;                                                            // [kSubPts][kMaxNb]

    const int tid = threadIdx.x, lane = tid & 31, warp = tid >> 5;
    for (int bi = blockIdx.x; bi < P.nbatches; bi += gridDim.x) {
        const Batch B = P.batches[bi];
        int n1, n2, n3;
        unpack_dims(B.dims, n1, n2, n3);
        const int ns = B.nslots, nb = B.nb, npb = n1 * n2 * n3;
        const int npad = (nb + 31) & ~31;
        __syncthreads();
        for (int s = tid; s < ns; s += kThreads) {
            Slot S = P.slots[B.slot0 + s];
            sl[s] = {S.atom, S.species, S.orb_off, S.norb, {S.d0[0], S.d0[1], S.d0[2]}};
        }
        for (int e = tid; e < ns * ns; e += kThreads) tbl[e] = P.tbl[B.tbl + tbl_index(e / ns, e % ns, ns)];
        __syncthreads();
        for (int s = tid; s < ns; s += kThreads)
            for (int o = 0; o < sl[s].norb; ++o) {
                oslot[sl[s].orb_off + o] = (unsigned char)s;
                oidx[sl[s].orb_off + o] = (unsigned char)o;
            }
        for (int p0 = 0; p0 < npb; p0 += kSubPts) {
            const int np = min(kSubPts, npb - p0);
            __syncthreads();
            // orbital values of every (point, slot) of the sub-batch; zero padding columns
            for (int w = tid; w < np * ns; w += kThreads) {
                const int p = w / ns, s = w - p * ns;
                const int lp = p0 + p;
                const int c = lp % n3, b = (lp / n3) % n2, a = lp / (n3 * n2);
                double off[3];
                point_offset64(P, a, b, c, off);
                T *row = Phi + p * kMaxNb + sl[s].orb_off;
                if constexpr (sizeof(T) == 8) {
                    eval_orbitals<double, false>(P, sl[s].species, sl[s].d0[0] + off[0], sl[s].d0[1] + off[1],
                                                 sl[s].d0[2] + off[2], [&](int o, double v) { row[o] = v; });
                } else {
                    float hx, lx, hy, ly, hz, lz, ox, oxl, oy, oyl, oz, ozl;
                    split_f32(sl[s].d0[0], hx, lx); split_f32(off[0], ox, oxl);
                    split_f32(sl[s].d0[1], hy, ly); split_f32(off[1], oy, oyl);
                    split_f32(sl[s].d0[2], hz, lz); split_f32(off[2], oz, ozl);
                    float dx = (hx + ox) + (lx + oxl), dy = (hy + oy) + (ly + oyl), dz = (hz + oz) + (lz + ozl);
                    eval_orbitals<float, false>(P, sl[s].species, dx, dy, dz, [&](int o, float v) { row[o] = v; });
                }
            }
            for (int w = tid; w < np * (npad - nb); w += kThreads) {
                const int p = w / (npad - nb), q = w - p * (npad - nb);
                Phi[p * kMaxNb + nb + q] = T(0);
            }
            for (int p = tid; p < np; p += kThreads) {
                const int lp = p0 + p;
                const int c = lp % n3, b = (lp / n3) % n2, a = lp / (n3 * n2);
                const int64_t g = ((int64_t)(B.i0 + a) * P.grid[1] + (B.j0 + b)) * P.grid[2] + (B.k0 + c);
                Vs[p] = (T)V[g];
            }
            __syncthreads();
            // upper-triangular 32x32 tiles; each warp owns whole tiles
            const int nt = npad / 32;
            const int ntp = nt * (nt + 1) / 2;
            const int ty = lane >> 3, tx = lane & 7;
            for (int tp = warp; tp < ntp; tp += kThreads / 32) {
                int ti = 0, rem = tp;
                while (rem >= nt - ti) { rem -= nt - ti; ++ti; }
                const int tj = ti + rem;
                T acc[8][4];
#pragma unroll
                for (int i = 0; i < 8; ++i)
#pragma unroll
                    for (int j = 0; j < 4; ++j) acc[i][j] = T(0);
                const int r0 = ti * 32 + ty * 8, c0 = tj * 32 + tx * 4;
                for (int p = 0; p < np; ++p) {
                    const T *row = Phi + p * kMaxNb;
                    const T v = Vs[p];
                    T ra[8], cb[4];
#pragma unroll
                    for (int i = 0; i < 8; ++i) ra[i] = row[r0 + i];
#pragma unroll
                    for (int j = 0; j < 4; ++j) cb[j] = v * row[c0 + j];
#pragma unroll
                    for (int i = 0; i < 8; ++i)
#pragma unroll
                        for (int j = 0; j < 4; ++j) acc[i][j] = fma(ra[i], cb[j], acc[i][j]);
                }
                const bool diag = (ti == tj);
#pragma unroll
                for (int i = 0; i < 8; ++i) {
                    const int mu = r0 + i;
                    if (mu >= nb) continue;
                    const int a = oslot[mu], oa = oidx[mu];
#pragma unroll
                    for (int j = 0; j < 4; ++j) {
                        const int nu = c0 + j;
                        if (nu >= nb) continue;
                        const int b = oslot[nu], ob = oidx[nu];
                        scatter_elem(H, tbl, ns, a, oa, sl[a].norb, b, ob, sl[b].norb, (double)acc[i][j] * P.dV, diag);
                    }
                }
            }
        }
    }
}

// Fill each non-canonical block with the transpose of its canonical partner.
__global__ void k_mirror(Plan P, double *H)
{
    const int64_t nb = P.nblocks;
    for (int64_t b = blockIdx.x; b < nb; b += gridDim.x) {
        const int pb = P.partner[b];
        const int64_t off = P.blk_off[b], poff = P.blk_off[pb];
        const int rows = P.blk_rows[b];
        const int cols = (int)((P.blk_off[b + 1] - off) / rows);
        // canonical = key <= partner key; the store is key-sorted, so canonical <=> b <= pb.
        // A self-partner block (b == pb) holds its upper triangle; copy it to the lower one.
        if (b < pb) continue;
        for (int e = threadIdx.x; e < rows * cols; e += blockDim.x) {
            const int mu = e / cols, nu = e - mu * cols;
            if (b == pb && mu <= nu) continue;
            H[off + e] = H[poff + nu * rows + mu];
        }
    }
}

template <typename T, bool RHO, bool FORCE>
__global__ void __launch_bounds__(kThreads, 1)
    k_rho_force_simt(Plan P, const double *__restrict__ V, const double *__restrict__ DM, double *rho, double *F,
                     double *dLde)
{
    extern __shared__ __align__(16) unsigned char smem[];
    SlotSh *sl = reinterpret_cast<SlotSh *>(smem);
    int *tbl = reinterpret_cast<int *>(sl + kMaxSlots);
    unsigned char *oslot = reinterpret_cast<unsigned char *>(tbl + kMaxSlots * kMaxSlots);
    unsigned char *oidx = oslot + kMaxNb;
    double *fsl = reinterpret_cast<double *>(oidx + kMaxNb);   // [kMaxSlots][3] force partials
    double *rhos = fsl + 3 * kMaxSlots;                         // [kRhoPts]
    T *Phi = reinterpret_cast<T *>(rhos + kRhoPts);             // [np_sub][npad]; Psi after the product
    T *Ds = Phi + kRhoTile;                                     // [2][kDChunk][npad]

    const int tid = threadIdx.x;
    // strain derivative: [0..8] Sum V grad_a phi . Psi d_b, [9] Sum V rho (this thread)
    double sacc[10];
#pragma unroll
    for (int k = 0; k < 10; ++k) sacc[k] = 0.0;
    for (int bi = blockIdx.x; bi < P.nbatches; bi += gridDim.x) {
        const Batch B = P.batches[bi];
        int n1, n2, n3;
        unpack_dims(B.dims, n1, n2, n3);
        const int ns = B.nslots, nb = B.nb, npb = n1 * n2 * n3;
        const int npad = (nb + 7) & ~7;
        // Psi = Phi D tiling: thread (tp, tc) owns points 4 tp .. 4 tp + 3 and columns
        // 8 tc .. 8 tc + 7; a sub-batch has as many points as the 256 threads cover, so every
        // multiply-add of a sub-batch lies inside the padded orbital range
        const int ncg = npad > 0 ? npad / 8 : 1;
        const int ngrp = kThreads / ncg;
        const int nsub = min(kRhoPts, 4 * ngrp);
        __syncthreads();
        for (int s = tid; s < ns; s += kThreads) {
            Slot S = P.slots[B.slot0 + s];
            sl[s] = {S.atom, S.species, S.orb_off, S.norb, {S.d0[0], S.d0[1], S.d0[2]}};
        }
        for (int e = tid; e < ns * ns; e += kThreads) tbl[e] = P.tbl[B.tbl + tbl_index(e / ns, e % ns, ns)];
        if (FORCE)
            for (int e = tid; e < 3 * ns; e += kThreads) fsl[e] = 0.0;
        __syncthreads();
        for (int s = tid; s < ns; s += kThreads)
            for (int o = 0; o < sl[s].norb; ++o) {
                oslot[sl[s].orb_off + o] = (unsigned char)s;
                oidx[sl[s].orb_off + o] = (unsigned char)o;
            }
        // D rows k0 .. k0 + kDChunk - 1 (all columns; zero outside the batch) into registers
        T dv[kDRegs];
        auto gather = [&](int k0) {
#pragma unroll
            for (int q = 0; q < kDRegs; ++q) {
                const int e = tid + q * kThreads;
                const int kr = e / npad, nu = e - kr * npad;
                const int mu = k0 + kr;
                T v = T(0);
                if (kr < kDChunk && mu < nb && nu < nb) {
                    const int a = oslot[mu], b = oslot[nu];
                    const int t = tbl[a * ns + b];
                    if (t >= 0) v = (T)DM[(t >> 1) + oidx[mu] * sl[b].norb + oidx[nu]];
                }
                dv[q] = v;
            }
        };
        auto stage = [&](T *dst) {
#pragma unroll
            for (int q = 0; q < kDRegs; ++q) {
                const int e = tid + q * kThreads;
                if (e < kDChunk * npad) dst[e] = dv[q];
            }
        };
        for (int p0 = 0; p0 < npb; p0 += nsub) {
            const int np = min(nsub, npb - p0);
            __syncthreads();
            for (int w = tid; w < nsub * ns; w += kThreads) {
                const int p = w / ns, s = w - p * ns;
                T *row = Phi + p * npad + sl[s].orb_off;
                if (p >= np) {
                    for (int o = 0; o < sl[s].norb; ++o) row[o] = T(0);
                    continue;
                }
                const int lp = p0 + p;
                const int c = lp % n3, b = (lp / n3) % n2, a = lp / (n3 * n2);
                double off[3];
                point_offset64(P, a, b, c, off);
                if constexpr (sizeof(T) == 8) {
                    eval_orbitals<double, false>(P, sl[s].species, sl[s].d0[0] + off[0], sl[s].d0[1] + off[1],
                                                 sl[s].d0[2] + off[2], [&](int o, double v) { row[o] = v; });
                } else {
                    float hx, lx, hy, ly, hz, lz, ox, oxl, oy, oyl, oz, ozl;
                    split_f32(sl[s].d0[0], hx, lx); split_f32(off[0], ox, oxl);
                    split_f32(sl[s].d0[1], hy, ly); split_f32(off[1], oy, oyl);
                    split_f32(sl[s].d0[2], hz, lz); split_f32(off[2], oz, ozl);
                    float dx = (hx + ox) + (lx + oxl), dy = (hy + oy) + (ly + oyl), dz = (hz + oz) + (lz + ozl);
                    eval_orbitals<float, false>(P, sl[s].species, dx, dy, dz, [&](int o, float v) { row[o] = v; });
                }
            }
            for (int w = tid; w < nsub * (npad - nb); w += kThreads) {
                const int p = w / (npad - nb), q = w - p * (npad - nb);
                Phi[p * npad + nb + q] = T(0);
            }
            for (int p = tid; p < nsub; p += kThreads) rhos[p] = 0.0;
            const bool gemm = tid < ngrp * ncg && npad > 0;
            const int tp = tid / ncg, tc = tid - (tid / ncg) * ncg;
            T acc[4][8];
#pragma unroll
            for (int i = 0; i < 4; ++i)
#pragma unroll
                for (int j = 0; j < 8; ++j) acc[i][j] = T(0);
            // the next chunk's D values are loaded while the current chunk is multiplied
            if (npad > 0) {
                gather(0);
                stage(Ds);
            }
            for (int k0 = 0, buf = 0; k0 < npad; k0 += kDChunk, buf ^= 1) {
                __syncthreads();
                const bool more = k0 + kDChunk < npad;
                if (more) gather(k0 + kDChunk);
                const T *D0 = Ds + buf * kDChunk * npad;
                const int kmax = min(kDChunk, npad - k0);
                if (gemm && 4 * tp < nsub)
                    for (int kr = 0; kr < kmax; ++kr) {
                        T pa[4], db[8];
#pragma unroll
                        for (int i = 0; i < 4; ++i) pa[i] = Phi[(tp * 4 + i) * npad + k0 + kr];
#pragma unroll
                        for (int j = 0; j < 8; ++j) db[j] = D0[kr * npad + tc * 8 + j];
#pragma unroll
                        for (int i = 0; i < 4; ++i)
#pragma unroll
                            for (int j = 0; j < 8; ++j) acc[i][j] = fma(pa[i], db[j], acc[i][j]);
                    }
                if (more) stage(Ds + (buf ^ 1) * kDChunk * npad);
            }
            __syncthreads();
            if (gemm && 4 * tp < nsub)
#pragma unroll
                for (int i = 0; i < 4; ++i)
#pragma unroll
                    for (int j = 0; j < 8; ++j) Phi[(tp * 4 + i) * npad + tc * 8 + j] = acc[i][j];
            const T *Psi = Phi;
            __syncthreads();
            // per (point, slot): rho and force contributions with recomputed (grad) orbitals
            for (int w = tid; w < np * ns; w += kThreads) {
                const int p = w / ns, s = w - p * ns;
                const int lp = p0 + p;
                const int c = lp % n3, b = (lp / n3) % n2, a = lp / (n3 * n2);
                double off[3];
                point_offset64(P, a, b, c, off);
                const T *prow = Psi + p * npad + sl[s].orb_off;
                T racc = T(0), gx = T(0), gy = T(0), gz = T(0);
                T ddx, ddy, ddz;   // displacement r - tau - R of this (point, atom image)
                if constexpr (sizeof(T) == 8) {
                    const double dx = sl[s].d0[0] + off[0], dy = sl[s].d0[1] + off[1], dz = sl[s].d0[2] + off[2];
                    ddx = dx; ddy = dy; ddz = dz;
                    if (FORCE)
                        eval_orbitals<double, true>(P, sl[s].species, dx, dy, dz,
                                                    [&](int o, double v, double x, double y, double z) {
                                                        const double q = prow[o];
                                                        racc += v * q; gx += x * q; gy += y * q; gz += z * q;
                                                    });
                    else
                        eval_orbitals<double, false>(P, sl[s].species, dx, dy, dz,
                                                     [&](int o, double v) { racc += v * prow[o]; });
                } else {
                    float hx, lx, hy, ly, hz, lz, ox, oxl, oy, oyl, oz, ozl;
                    split_f32(sl[s].d0[0], hx, lx); split_f32(off[0], ox, oxl);
                    split_f32(sl[s].d0[1], hy, ly); split_f32(off[1], oy, oyl);
                    split_f32(sl[s].d0[2], hz, lz); split_f32(off[2], oz, ozl);
                    float dx = (hx + ox) + (lx + oxl), dy = (hy + oy) + (ly + oyl), dz = (hz + oz) + (lz + ozl);
                    ddx = dx; ddy = dy; ddz = dz;
                    if (FORCE)
                        eval_orbitals<float, true>(P, sl[s].species, dx, dy, dz,
                                                   [&](int o, float v, float x, float y, float z) {
                                                       const float q = prow[o];
                                                       racc += v * q; gx += x * q; gy += y * q; gz += z * q;
                                                   });
                    else
                        eval_orbitals<float, false>(P, sl[s].species, dx, dy, dz,
                                                    [&](int o, float v) { racc += v * prow[o]; });
                }
                if (RHO) atomicAdd(&rhos[p], (double)racc);
                if (FORCE) {
                    const int64_t g = ((int64_t)(B.i0 + a) * P.grid[1] + (B.j0 + b)) * P.grid[2] + (B.k0 + c);
                    const double w2 = V[g];
                    if (F) {
                        atomicAdd(&fsl[3 * s + 0], w2 * (double)gx);
                        atomicAdd(&fsl[3 * s + 1], w2 * (double)gy);
                        atomicAdd(&fsl[3 * s + 2], w2 * (double)gz);
                    }
                    if (dLde) {
                        const double gg[3] = {w2 * (double)gx, w2 * (double)gy, w2 * (double)gz};
                        const double dd[3] = {(double)ddx, (double)ddy, (double)ddz};
#pragma unroll
                        for (int u = 0; u < 3; ++u)
#pragma unroll
                            for (int v = 0; v < 3; ++v) sacc[3 * u + v] += gg[u] * dd[v];
                        sacc[9] += w2 * (double)racc;
                    }
                }
            }
            __syncthreads();
            if (RHO)
                for (int p = tid; p < np; p += kThreads) {
                    const int lp = p0 + p;
                    const int c = lp % n3, b = (lp / n3) % n2, a = lp / (n3 * n2);
                    const int64_t g = ((int64_t)(B.i0 + a) * P.grid[1] + (B.j0 + b)) * P.grid[2] + (B.k0 + c);
                    rho[g] = rhos[p];
                }
        }
        if (FORCE && F) {
            __syncthreads();
            for (int e = tid; e < 3 * ns; e += kThreads) {
                const int s = e / 3, q = e - 3 * s;
                atomicAdd(&F[3 * sl[s].atom + q], 2.0 * P.dV * fsl[e]);
            }
        }
    }
    if (FORCE && dLde) {
        // dL/deps_ab = 2 dV Sum V grad_a phi . Psi d_b + delta_ab dV Sum V rho
#pragma unroll
        for (int k = 0; k < 10; ++k)
#pragma unroll
            for (int m = 16; m > 0; m >>= 1) sacc[k] += __shfl_xor_sync(0xffffffffu, sacc[k], m);
        if ((tid & 31) == 0) {
            for (int k = 0; k < 9; ++k)
                atomicAdd(&dLde[k], 2.0 * P.dV * sacc[k] + ((k % 4) == 0 ? P.dV * sacc[9] : 0.0));
        }
    }
}

template <typename T>
size_t vlocal_smem()
{
    return sizeof(SlotSh) * kMaxSlots + sizeof(int) * kMaxSlots * kMaxSlots + 2 * kMaxNb + sizeof(T) * kSubPts +
           sizeof(T) * kSubPts * kMaxNb;
}

template <typename T>
size_t rho_smem()
{
    return sizeof(SlotSh) * kMaxSlots + sizeof(int) * kMaxSlots * kMaxSlots + 2 * kMaxNb +
           sizeof(double) * (3 * kMaxSlots + kRhoPts) + sizeof(T) * (kRhoTile + 2 * kDChunk * kMaxNb);
}

template <typename K>
cudaError_t launch_persistent(K kernel, size_t smem, int nsm, cudaStream_t s, const Plan &P, const double *a,
                              const double *b, double *c, double *d, int variant)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int grid = nsm;
    if (grid > P.nbatches) grid = P.nbatches;
    if (grid < 1) return cudaSuccess;
    (void)variant;
    kernel<<<grid, kThreads, smem, s>>>(P, a, b, c, d);
    return cudaGetLastError();
}

}  // namespace

cudaError_t launch_mirror(const Plan &P, double *H, cudaStream_t s)
{
    if (P.nblocks == 0) return cudaSuccess;
    int grid = (int)std::min<int64_t>(P.nblocks, 4096);
    k_mirror<<<grid, 128, 0, s>>>(P, H);
    return cudaGetLastError();
}

cudaError_t launch_vlocal_simt(const Plan &P, bool fp64, const double *V, double *H, cudaStream_t s, int nsm)
{
    if (P.nbatches == 0) return cudaSuccess;
    cudaError_t e;
    int grid = std::min(nsm, P.nbatches);
    if (fp64) {
        size_t smem = vlocal_smem<double>();
        e = cudaFuncSetAttribute(k_vlocal_simt<double>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_vlocal_simt<double><<<grid, kThreads, smem, s>>>(P, V, H);
    } else {
        size_t smem = vlocal_smem<float>();
        e = cudaFuncSetAttribute(k_vlocal_simt<float>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_vlocal_simt<float><<<grid, kThreads, smem, s>>>(P, V, H);
    }
    return cudaGetLastError();
}

template <typename T>
static cudaError_t launch_rf(const Plan &P, const double *V, const double *DM, double *rho, double *F, double *dLde,
                             cudaStream_t s, int nsm)
{
    size_t smem = rho_smem<T>();
    int grid = std::min(nsm, P.nbatches);
    cudaError_t e;
    const bool force = F || dLde;
    if (rho && force) {
        e = cudaFuncSetAttribute(k_rho_force_simt<T, true, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_rho_force_simt<T, true, true><<<grid, kThreads, smem, s>>>(P, V, DM, rho, F, dLde);
    } else if (rho) {
        e = cudaFuncSetAttribute(k_rho_force_simt<T, true, false>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_rho_force_simt<T, true, false><<<grid, kThreads, smem, s>>>(P, V, DM, rho, F, dLde);
    } else {
        e = cudaFuncSetAttribute(k_rho_force_simt<T, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
        k_rho_force_simt<T, false, true><<<grid, kThreads, smem, s>>>(P, V, DM, rho, F, dLde);
    }
    return cudaGetLastError();
}

cudaError_t launch_rho_force_simt(const Plan &P, bool fp64, const double *V, const double *DM, double *rho, double *F,
                                  double *dLde, cudaStream_t s, int nsm)
{
    if (P.nbatches == 0) return cudaSuccess;
    return fp64 ? launch_rf<double>(P, V, DM, rho, F, dLde, s, nsm) : launch_rf<float>(P, V, DM, rho, F, dLde, s, nsm);
}

}  // namespace gint
