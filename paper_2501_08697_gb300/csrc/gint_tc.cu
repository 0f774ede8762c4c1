// tcgen05 tensor-core kernels of libgint: the split-precision grid integrations.
//
// The per-batch contractions (Sec. IV.B: "parallel matrix operations" over partitions of the
// real-space grid) run on the 5th-generation tensor cores:
//   vlocal      P_b = Phi_b^T diag(V) Phi_b dV      M = N = orbitals of the batch, K = points
//   rho/force   Psi_b = Phi_b D_b                   M = points, N = K = orbitals of the batch
// Each FP32 operand x is split into terms (hi + lo for TF32x3 and BF16x3, hi + mid + lo for
// BF16x6); the products of total order <= 1 (TF32x3, BF16x3) or <= 2 (BF16x6) accumulate in
// FP32 in tensor memory (TMEM); the cross-batch sums (block store, rho(r), forces) are FP64.
//
// One persistent CTA per SM, 20 warps (5 per SM sub-partition, which leaves 96 registers a
// thread; the producers carry most of the CUDA-core work):
//   warps 0-10 producers: orbital values (FP32, spline x solid harmonic) into an FP32 staging
//              tile, then split into the canonical K-major no-swizzle shared-memory layout
//              (8-row x 16-byte core matrices; the K-direction core-matrix stride is padded
//              to 144 bytes so 16-byte stores from a warp spread over all banks).
//   warp 11    one thread issues the MMAs of each chunk once the producers have arrived on
//              the stage's barrier, and commits them to the stage's and accumulator's barriers.
//   warps 12-19 epilogue: tcgen05.ld of the accumulator (warp w reads TMEM lanes 32(w%4)..;
//              the two warps of a lane quadrant share the columns or the atom images),
//              then the FP64 scatter into the block store (vlocal) or rho(r)/force (rho).
// Accumulators are double-buffered in TMEM so the epilogue of batch i overlaps the MMAs of
// batch i+1.  No FP64 arithmetic runs in the hot loops (GB300's FP64 rate is 1/64 of FP32):
// offsets come as FP32 hi/lo pairs, dV is folded into the FP32 operand, FP32 -> FP64 for the
// reductions (red.global.add.f64, no return value) is done with integer bit operations, and the
// density matrix is read as FP32.
// Every mbarrier wait is bounded (clock64 budget); a wait that runs out records
// GINT_ETIMEOUT in the status word and the CTA drains and exits without deadlock.
#include <cuda_bf16.h>

#include "gint_device.cuh"
#include "gint_tcgen05.cuh"

namespace gint {
namespace {

constexpr int kProd = 352;        // producer threads (warps 0-10)
constexpr int kMma = kProd;       // the MMA-issue thread (warp 11)
constexpr int kEpi0 = kProd + 32; // first epilogue thread (warp 12: TMEM lane quadrant = warp % 4)
constexpr int kEpi = 256;         // epilogue threads (two warps per TMEM lane quadrant)
constexpr int kThreadsTC = kEpi0 + kEpi;
constexpr int kWin = 32;          // epilogue window (columns) of the rho kernel
constexpr int kVTblR = 28;        // atom images of a batch whose slot-pair table the rho kernel keeps in shared memory

// ------------------------------------------------------------------ shared batch metadata
// An atom image of the batch in shared memory: the first 16 bytes and dh/dl as in Slot, so
// they can be copied asynchronously in 8-byte pieces.
struct PSlot {
    int atom, species, off, norb;
    float dh[3], dl[3];
};
static_assert(sizeof(PSlot) == 40, "PSlot layout");
static_assert(offsetof(TSlot, dh) == 16 && sizeof(TSlot) == 40, "TSlot layout: copied into PSlot as is");

__device__ __forceinline__ void unpack(int dims, int &n1, int &n2, int &n3)
{
    n1 = dims & 255;
    n2 = (dims >> 8) & 255;
    n3 = (dims >> 16) & 255;
}

// structure info of the current batch, reloaded only when the structure id changes (a CTA's
// contiguous batch range spans few structures)
struct SInfoCache {
    int sid;
    SInfo v;
    __device__ __forceinline__ SInfoCache(const SInfo &si0) : sid(-1), v(si0) {}
    __device__ __forceinline__ SInfo get(const Batch &B, const SInfo *sis)
    {
        if (sis) {
            const int id = (int)((unsigned)B.dims >> 24);
            if (id != sid) {
                sid = id;
                v = sis[id];
            }
        }
        return v;
    }
};

// The batches of this CTA, in order: per segment (the whole list, or one structure of a
// multi-structure job) one contiguous range.  Contiguous ranges keep the CTAs that run at the
// same time on distant parts of a cell, so their FP64 atomics rarely meet on one block; the
// segments keep all CTAs on the same structure at about the same time.
struct CtaRange {
    const int2 *rng;
    int npart, nseg, seg, cur, end;
    __device__ __forceinline__ CtaRange(const Plan &P) : rng(P.rng), npart(P.npart), nseg(P.nseg), seg(0)
    {
        if (rng) {
            const int2 r = rng[blockIdx.x];
            cur = r.x;
            end = r.y;
        } else {
            nseg = 1;
            cur = (int)((int64_t)P.nbatches * blockIdx.x / gridDim.x);
            end = (int)((int64_t)P.nbatches * (blockIdx.x + 1) / gridDim.x);
        }
    }
    __device__ __forceinline__ bool next(int &bi)
    {
        while (cur >= end) {
            if (++seg >= nseg) return false;
            const int2 r = rng[seg * npart + blockIdx.x];
            cur = r.x;
            end = r.y;
        }
        bi = cur++;
        return true;
    }
};

// slots and point offsets of batch B into shared memory (called by the threads of one role)
__device__ __forceinline__ void load_geom(const Plan &P, const SInfo &SI, const Batch &B, PSlot *ps, float *poff,
                                          int tid, int nthr)
{
    for (int s = tid; s < B.nslots; s += nthr) {
        const TSlot &S = P.tslots[B.slot0 + s];
        PSlot q;
        q.species = S.species;
        q.off = S.orb_off;
        q.norb = S.norb;
        q.atom = S.atom;
        for (int c = 0; c < 3; ++c) {
            q.dh[c] = S.dh[c];
            q.dl[c] = S.dl[c];
        }
        ps[s] = q;
    }
    int n1, n2, n3;
    unpack(B.dims, n1, n2, n3);
    const int np = n1 * n2 * n3;
    for (int p = tid; p < np; p += nthr) {
        const int c = p % n3, b = (p / n3) % n2, a = p / (n3 * n2);
        const float *t = SI.poff + ((a * kPoffDim + b) * kPoffDim + c) * 6;
#pragma unroll
        for (int q = 0; q < 6; ++q) poff[6 * p + q] = __ldg(t + q);
    }
}

// Start copying the geometry of batch B (its atom images, point offsets and, when vd is not
// null, the potential at its points) into shared memory; the calling role waits with
// cp_async_wait_all and a barrier before reading it.
__device__ __forceinline__ void geom_async(const Plan &P, const SInfo *sis, const SInfo &si0, const Batch &B,
                                           PSlot *ps, float *poff, double *vd, int tid, int nthr)
{
    const double *V = si0.V;
    const float *ptab = si0.poff;
    int g1 = si0.grid[1], g2 = si0.grid[2];
    if (sis) {
        const SInfo &S = sis[(unsigned)B.dims >> 24];
        V = S.V;
        ptab = S.poff;
        g1 = S.grid[1];
        g2 = S.grid[2];
    }
    for (int w = tid; w < B.nslots * 5; w += nthr) {
        const int s = w / 5, part = w - 5 * s;
        const char *src = reinterpret_cast<const char *>(P.tslots + B.slot0 + s);
        char *dst = reinterpret_cast<char *>(ps + s);
        cp_async8(dst + 8 * part, src + 8 * part);
    }
    int n1, n2, n3;
    n1 = B.dims & 255;
    n2 = (B.dims >> 8) & 255;
    n3 = (B.dims >> 16) & 255;
    const int np = n1 * n2 * n3;
    for (int w = tid; w < np * 4; w += nthr) {
        const int p = w >> 2, part = w & 3;
        const int c = p % n3, b = (p / n3) % n2, a = p / (n3 * n2);
        if (part < 3) {
            cp_async8(poff + 6 * p + 2 * part, ptab + ((a * kPoffDim + b) * kPoffDim + c) * 6 + 2 * part);
        } else if (vd) {
            cp_async8(vd + p, V + ((int64_t)(B.i0 + a) * g1 + (B.j0 + b)) * g2 + (B.k0 + c));
        }
    }
    cp_async_commit();
}

__device__ __forceinline__ void cp_async4(void *dst, const void *src)
{
    asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(su32(dst)), "l"(src) : "memory");
}

// The density kernel's batch metadata (atom images, point offsets, padded K offsets and, for at
// most kVTbl images, the slot-pair split-store table) copied asynchronously into one half of
// the producers' double-buffered arrays; the caller waits with cp_async_wait_all and a barrier.
__device__ __forceinline__ void geom_async_rho(const Plan &P, const SInfo *sis, const SInfo &si0, const Batch &B,
                                               PSlot *ps, float *poff, int *koffs, int *tbls, int tid, int nthr)
{
    geom_async(P, sis, si0, B, ps, poff, nullptr, tid, nthr);
    const int ns = B.nslots;
    for (int s = tid; s < ns; s += nthr) cp_async4(koffs + s, P.koff + B.slot0 + s);
    if (ns <= kVTblR)
        for (int e = tid; e < ns * ns; e += nthr) cp_async4(tbls + e, P.tbl2 + B.tbl + e);
    cp_async_commit();
}

__device__ __forceinline__ void disp(const PSlot &s, const float *po, float &dx, float &dy, float &dz)
{
    dx = (s.dh[0] + po[0]) + (s.dl[0] + po[3]);
    dy = (s.dh[1] + po[1]) + (s.dl[1] + po[4]);
    dz = (s.dh[2] + po[2]) + (s.dl[2] + po[5]);
}

// centre of a batch relative to its origin point and the radius of a sphere about it that holds
// all its points (upper bound), from the grid step vectors
__device__ __forceinline__ void batch_sphere(const SInfo &SI, int n1, int n2, int n3, float *bc, float &R)
{
    const float *h = SI.hstep;
    const float f[3] = {0.5f * (n1 - 1), 0.5f * (n2 - 1), 0.5f * (n3 - 1)};
    float r = 0.f;
#pragma unroll
    for (int c = 0; c < 3; ++c) bc[c] = __fadd_rn(__fadd_rn(__fmul_rn(f[0], h[c]), __fmul_rn(f[1], h[3 + c])), __fmul_rn(f[2], h[6 + c]));
#pragma unroll
    for (int i = 0; i < 3; ++i)
        r = __fadd_rn(r, __fmul_rn(f[i], __fsqrt_rn(__fadd_rn(__fadd_rn(__fmul_rn(h[3 * i], h[3 * i]), __fmul_rn(h[3 * i + 1], h[3 * i + 1])),
                                                           __fmul_rn(h[3 * i + 2], h[3 * i + 2])))));
    R = __fadd_rn(__fmul_rn(r, 1.0001f), 1e-6f);
}

__device__ __forceinline__ int64_t grid_index(const SInfo &SI, const Batch &B, int p, int n2, int n3)
{
    const int c = p % n3, b = (p / n3) % n2, a = p / (n3 * n2);
    return ((int64_t)(B.i0 + a) * SI.grid[1] + (B.j0 + b)) * SI.grid[2] + (B.k0 + c);
}


__device__ __forceinline__ void load_species(const Plan &P, SpecSh *spec, int tid)
{
    if (tid < P.nspecies) {
        const DevSpecies &D = P.sp[tid];
        SpecSh q;
        q.nrad = D.nrad;
        q.nint = D.nint;
        q.coef_off = D.coef_off;
        int lp = 0;
        for (int r = 0; r < D.nrad; ++r) lp |= D.l[r] << (2 * r);
        q.lpack = lp;
        q.rcut2 = D.rcut_f * D.rcut_f;
        q.inv_dr = D.inv_dr_f;
        q.shape = shape_of(D.nrad, lp);
        q.env_off = D.env_off;
        spec[tid] = q;
    }
}

// ====================================================================== vlocal
// TMEM accumulators: a batch takes tile 0 (rows 0..127, N = npad columns) and, with more than
// 128 orbitals, tile 1 (rows 128.., N = npad - 128: only the columns of the upper triangle)
// right after it.  Consecutive batches of a CTA take consecutive column ranges of the 512-column
// memory (a ring), starting again from column 0 when a batch would not fit: two batches are in
// flight whenever their widths add up to 512 or less, and the MMA waits for the epilogue of the
// previous batch only when the ring wraps onto it.
struct TmemRing {
    int s = 0, w = 0;   // base column and width of the previous batch
    // base column of the next batch (npad orbitals, nb > 128 with tile 1); overlap: it wraps
    // onto the previous batch's columns
    __device__ __forceinline__ int next(int npad, int nb, bool &overlap)
    {
        const int W = npad + (nb > 128 ? npad - 128 : 0);
        int b = s + w;
        if (b + W > kTmemCols) b = 0;
        overlap = b == 0 && w > 0 && s < W;
        s = b;
        w = W;
        return b;
    }
};
// The vlocal epilogue keeps the batch's slot-pair table in shared memory when the batch has
// at most kVTbl atom images (nearly all batches), otherwise it reads it from global memory.
constexpr int kVTbl = 28;

template <class S>
struct VSmem {
    static constexpr int KC = S::KCM * S::CG;             // points per chunk
    static constexpr int ROWS = kMaxNb;                   // orbitals per batch
    static constexpr int ARR = arr_bytes<S>(256);         // one operand term (tile 1 reads rows 128..255)
    static constexpr int STAGE = 2 * S::NT * ARR;         // A terms then B terms
    // stages per scheme: with one, the chunk's MMAs overlap the next chunk's orbital
    // evaluation into the staging tile, which comes before the stage is rewritten
    static constexpr int NSTAGE = S::VSTAGES;
    static constexpr int OFF_STG = NSTAGE * STAGE;                          // float [256][KC]
    static constexpr int OFF_PSLOT = OFF_STG + ROWS * KC * 4;               // PSlot[2][64]
    static constexpr int OFF_POFF = OFF_PSLOT + 2 * kMaxSlots * (int)sizeof(PSlot);  // float [2][128][6]
    static constexpr int OFF_V = OFF_POFF + 2 * kMaxBatchPts * 6 * 4;       // float [128]: V dV of the batch
    static constexpr int OFF_TBL = OFF_V + kMaxBatchPts * 4;                // int [kVTbl^2]
    static constexpr int OFF_INFO = OFF_TBL + kVTbl * kVTbl * 4;            // int [256]: slot | o << 8 | norb << 16
    static constexpr int EXPB = S::HALF ? 2 * kMaxNb * 2 : 0;              // (fp16 scaling only)
    static constexpr int OFF_PEXP = OFF_INFO + kMaxNb * 4;                  // short [2][256]: producers' A, B exponents
    static constexpr int OFF_EEXP = OFF_PEXP + EXPB;                        // short [2][256]: epilogue's copy
    static constexpr int OFF_TILE = OFF_EEXP + EXPB;                        // float [8][32][33]
    static constexpr int OFF_BAR = OFF_TILE + 8 * 32 * 33 * 4;              // 16 mbarriers
    static constexpr int OFF_MISC = OFF_BAR + 16 * 8;                       // tmem base, flags
    static constexpr int OFF_SPEC = OFF_MISC + 64;                          // SpecSh[kMaxSpecies]
    static constexpr int TOTAL = OFF_SPEC + kMaxSpecies * (int)sizeof(SpecSh);
};

template <class S>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_vlocal_tc(Plan P, SInfo si0, const SInfo *__restrict__ sis)
{
    using L = VSmem<S>;
    constexpr int KC = L::KC, NS = L::NSTAGE;
    constexpr int SBO = S::KCM * kLBO;
    extern __shared__ __align__(1024) unsigned char sm[];
    float *stg = reinterpret_cast<float *>(sm + L::OFF_STG);
    PSlot *psb = reinterpret_cast<PSlot *>(sm + L::OFF_PSLOT);
    float *poffb = reinterpret_cast<float *>(sm + L::OFF_POFF);
    float *vs = reinterpret_cast<float *>(sm + L::OFF_V);
    int *tbls = reinterpret_cast<int *>(sm + L::OFF_TBL);
    int *info = reinterpret_cast<int *>(sm + L::OFF_INFO);
    short *pexp = reinterpret_cast<short *>(sm + L::OFF_PEXP), *eexp = reinterpret_cast<short *>(sm + L::OFF_EEXP);
    float *tiles = reinterpret_cast<float *>(sm + L::OFF_TILE);
    SpecSh *spec = reinterpret_cast<SpecSh *>(sm + L::OFF_SPEC);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::OFF_BAR);
    uint64_t *empty = bars, *accfull = bars + 2, *accempty = bars + 4, *fin = bars + 6, *full = bars + 8;
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(sm + L::OFF_MISC);
    volatile int *pflag = reinterpret_cast<volatile int *>(sm + L::OFF_MISC + 4);
    volatile int *eflag = reinterpret_cast<volatile int *>(sm + L::OFF_MISC + 8);

    const int tid = threadIdx.x, warp = tid >> 5;
    load_species(P, spec, tid);
    if (tid == 0) {
        mbar_init(&empty[0], 1);
        mbar_init(&empty[1], 1);
        mbar_init(&accfull[0], 1);
        mbar_init(&accfull[1], 1);
        mbar_init(&accempty[0], kEpi);
        mbar_init(&accempty[1], kEpi);
        mbar_init(fin, 1);
        mbar_init(&full[0], 1);
        mbar_init(&full[1], 1);
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

    if (tid < kProd) {
        // ------------------------------------------------------------ producers
        const int pt = tid;
        int g = 0;  // chunk counter (stage = g & 1)
        bool ok = true;
        SInfoCache sic(si0);
        // The geometry of the next batch is copied asynchronously into the other half of the
        // double-buffered slot / offset / potential arrays while this batch is computed.
        CtaRange cr(P);
        int bi = 0, cur = 0;
        bool have = cr.next(bi);
        if (have) geom_async(P, sis, si0, P.batches[bi], psb, poffb, nullptr, pt, kProd);
        for (; ok && have; have = cr.next(bi), cur ^= 1) {
            const Batch B = P.batches[bi];
            int n1, n2, n3;
            unpack(B.dims, n1, n2, n3);
            const int ns = B.nslots, nb = B.nb, npb = n1 * n2 * n3;
            const int npad = (nb + 15) & ~15;
            CtaRange peek = cr;
            int bn = 0;
            const bool more = peek.next(bn);
            const Batch Bn = P.batches[more ? bn : bi];
            const PSlot *ps = psb + cur * kMaxSlots;
            const float *poff = poffb + cur * kMaxBatchPts * 6;
            cp_async_wait_all();
            named_sync(1, kProd);   // this batch's geometry is in buffer cur; buffer cur ^ 1 is free
            if (nb == 0) {          // no orbital reaches this batch: nothing to add
                if (more) geom_async(P, sis, si0, Bn, psb + (cur ^ 1) * kMaxSlots, poffb + (cur ^ 1) * kMaxBatchPts * 6,
                                     nullptr, pt, kProd);
                continue;
            }
            const SInfo SI = sic.get(B, sis);
            const float dVf = (float)SI.dV;
            if constexpr (S::HALF) {
                // fp16 operands: row mu of A = phi_mu 2^eA(mu), row nu of B = V dV phi_nu 2^eB(nu),
                // with exponents per atom image from a bound on its |phi| over this batch, so
                // that the orbitals of distant images keep their relative accuracy (undone in
                // the epilogue)
                float bc[3], R;
                batch_sphere(SI, n1, n2, n3, bc, R);
                for (int s = pt; s < ns; s += kProd) {
                    const PSlot sl = ps[s];
                    const float m = phi_bound(P.env, spec[sl.species], sl.dh, sl.dl, bc, R);
                    const short ea = (short)scale_exp(m), eb = (short)scale_exp(SI.amax[0] * dVf * m);
                    for (int o = 0; o < sl.norb; ++o) {
                        pexp[sl.off + o] = ea;
                        pexp[kMaxNb + sl.off + o] = eb;
                    }
                }
            }
            // V dV of the batch's points (read here; the stages take the shared memory a
            // prefetched copy would need)
            for (int p = pt; p < kMaxBatchPts; p += kProd)
                vs[p] = p < npb ? d2f(__ldg(SI.V + grid_index(SI, B, p, n2, n3))) * dVf : 0.f;
            const int nch = (npb + KC - 1) / KC;
            for (int ch = 0; ch < nch && ok; ++ch, ++g) {
                const int stage = g % NS;
                // phase 1: orbital values at the chunk's points -> staging [row][KC]
                for (int w = pt; w < KC * ns; w += kProd) {
                    const int k = w % KC, s = w / KC;
                    const int p = ch * KC + k;
                    const PSlot sl = ps[s];
                    float *col = stg + sl.off * KC + k;
                    if (p < npb) {
                        float dx, dy, dz;
                        disp(sl, poff + 6 * p, dx, dy, dz);
                        eval_phi_any<!S::F16>(spec[sl.species], P.coef32, dx, dy, dz, [&](int o, float v) { col[o * KC] = v; });
                    } else {
                        for (int o = 0; o < sl.norb; ++o) col[o * KC] = 0.f;
                    }
                }
                if (ch == 0 && more)
                    geom_async(P, sis, si0, Bn, psb + (cur ^ 1) * kMaxSlots, poffb + (cur ^ 1) * kMaxBatchPts * 6,
                               nullptr, pt, kProd);
                if (g >= NS) ok = role_wait(&empty[stage], ((g / NS) - 1) & 1, P, pt, pflag, 1, kProd);
                else named_sync(1, kProd);
                if (!ok) break;
                // phase 2: split Phi (A) and V dV Phi (B) into the canonical layout
                unsigned char *base = sm + stage * L::STAGE;
                for (int w = pt; w < npad * S::KCM; w += kProd) {
                    const int kc = w % S::KCM, row = w / S::KCM;
                    // accumulator row of orbital `row`: tile 1 (orbitals 128..) takes the TMEM
                    // lane quadrants in reverse order, so its rows land in the quadrants with the
                    // fewest upper-triangle pieces of tile 0 and the epilogue warps share the
                    // scatter evenly
                    const int arow = row < 128 ? row : (row ^ 0x60);
                    unsigned char *da[S::NT], *db[S::NT];
#pragma unroll
                    for (int t = 0; t < S::NT; ++t) {
                        da[t] = base + t * L::ARR + cm_off<S>(arow, kc);
                        db[t] = base + (S::NT + t) * L::ARR + cm_off<S>(row, kc);
                    }
                    if (row < nb) {
                        float x[S::CG], y[S::CG];
                        float sa = 1.f, sb = 1.f;
                        if constexpr (S::HALF) {
                            sa = pow2i(pexp[row]);
                            sb = pow2i(pexp[kMaxNb + row]);
                        }
#pragma unroll
                        for (int i = 0; i < S::CG; ++i) {
                            x[i] = stg[row * KC + kc * S::CG + i];
                            y[i] = x[i] * vs[ch * KC + kc * S::CG + i];
                            if constexpr (S::HALF) {
                                x[i] *= sa;
                                y[i] *= sb;
                            }
                        }
                        split_store<S>(x, da);
                        split_store<S>(y, db);
                    } else {
                        zero_store<S>(da);
                        zero_store<S>(db);
                    }
                }
                fence_async_smem();
                named_sync(1, kProd);
                if (pt == 0) mbar_arrive(&full[stage]);   // chunk g is in shared memory
            }
        }
        cp_async_wait_all();   // no copy may be in flight when the CTA exits
    } else if (tid < kEpi0) {
        // ------------------------------------------------------------ MMA issue (one thread)
        // Follows the producers' chunk sequence: waits until chunk g is in stage g & 1 (and, at
        // a batch's first chunk, until the epilogue has released the accumulator), issues the
        // chunk's MMAs and commits them to the stage's and the accumulator's barriers.
        if (tid == kMma) {
            int g = 0, it = 0;
            bool ok = true;
            CtaRange cr(P);
            TmemRing ring;
            for (int bi = 0; ok && cr.next(bi);) {
                const Batch B = P.batches[bi];
                int n1, n2, n3;
                unpack(B.dims, n1, n2, n3);
                const int nb = B.nb, npb = n1 * n2 * n3;
                if (nb == 0) continue;
                const int npad = (nb + 15) & ~15;
                const int buf = it & 1;
                bool wrap;
                const int base = ring.next(npad, nb, wrap);
                const int nch = (npb + KC - 1) / KC;
                for (int ch = 0; ch < nch && ok; ++ch, ++g) {
                    const int stage = g % NS;
                    ok = !aborted(P) && mbar_wait(&full[stage], (g / NS) & 1, P.spin_limit);
                    if (ok && ch == 0 && it >= 2)   // the epilogue of batch it - 2 is done
                        ok = !aborted(P) && mbar_wait(&accempty[buf], ((it >> 1) - 1) & 1, P.spin_limit);
                    if (ok && ch == 0 && wrap)      // and of batch it - 1, whose columns this one reuses
                        ok = !aborted(P) && mbar_wait(&accempty[buf ^ 1], ((it - 1) >> 1) & 1, P.spin_limit);
                    if (!ok) {
                        report_timeout(P);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = su32(sm + stage * L::STAGE), b0 = a0 + S::NT * L::ARR;
#pragma unroll
                    for (int ks = 0; ks < S::KCM / 2; ++ks) {
                        for (int t = 0; t < (nb > 128 ? 2 : 1); ++t) {
                            const int N = t == 0 ? npad : npad - 128;
                            const uint32_t id = idesc<S>(128, N);
                            const uint32_t rowoff = t * 16 * SBO;
#pragma unroll
                            for (int q = 0; q < S::NPROD; ++q) {
                                const uint64_t da = sdesc(a0 + term(S::PA, q) * L::ARR + rowoff + ks * 2 * kLBO, SBO);
                                const uint64_t db = sdesc(b0 + term(S::PB, q) * L::ARR + rowoff + ks * 2 * kLBO, SBO);
                                const uint32_t acc = (ch == 0 && ks == 0 && q == 0) ? 0u : 1u;
                                umma<S::F16>(tmem + base + t * npad, da, db, id, acc);
                            }
                        }
                    }
                    umma_commit(&empty[stage]);
                    if (ch == nch - 1) umma_commit(&accfull[buf]);
                }
                ++it;
            }
            // wait (bounded) for every MMA this thread issued before TMEM is released
            umma_commit(fin);
            if (!mbar_wait(fin, 0, kDrainBudget)) report_timeout(P);
        }
    } else {
        // ------------------------------------------------------------ epilogue
        const int et = tid - kEpi0, ew = et >> 5, lane = et & 31;
        const int q = ew & 3, hh = ew >> 2;  // TMEM lane quadrant, column half
        int it = 0;
        SInfoCache sic(si0);
        CtaRange cr(P);
        TmemRing ring;
        for (int bi = 0; cr.next(bi);) {
            const Batch B = P.batches[bi];
            const int ns = B.nslots, nb = B.nb;
            const int npad = (nb + 15) & ~15;
            const int buf = it & 1;
            if (nb == 0) continue;
            bool wrap;
            const int base = ring.next(npad, nb, wrap);
            const SInfo SIe = sic.get(B, sis);
            double *H = SIe.H;
            const bool small = ns <= kVTbl;
            const int *tbl = P.tbl + B.tbl;
            named_sync(2, kEpi);
            if (small)
                for (int e = et; e < ns * ns; e += kEpi) {
                    // the scatter adds only for pairs a <= b: the upper triangle, which leads the
                    // table, is fetched, and the rest of the copy (row-major) is -1
                    const int a = e / ns, b = e - a * ns;
                    tbls[e] = b >= a ? __ldg(tbl + tbl_index(a, b, ns)) : -1;
                }
            float bc[3], R;
            if constexpr (S::HALF) {
                int n1, n2, n3;
                unpack(B.dims, n1, n2, n3);
                batch_sphere(SIe, n1, n2, n3, bc, R);
            }
            for (int s = et; s < ns; s += kEpi) {
                const TSlot &sl = P.tslots[B.slot0 + s];
                const int no = sl.norb, off = sl.orb_off;
                short ea = 0, eb = 0;
                if constexpr (S::HALF) {
                    // the producers' exponents of this image (same inputs, same rounded arithmetic)
                    const float dh[3] = {sl.dh[0], sl.dh[1], sl.dh[2]}, dl[3] = {sl.dl[0], sl.dl[1], sl.dl[2]};
                    const float m = phi_bound(P.env, spec[sl.species], dh, dl, bc, R);
                    ea = (short)scale_exp(m);
                    eb = (short)scale_exp(SIe.amax[0] * (float)SIe.dV * m);
                }
                for (int o = 0; o < no; ++o) {
                    info[off + o] = s | (o << 8) | (no << 16);
                    eexp[off + o] = ea;
                    eexp[kMaxNb + off + o] = eb;
                }
            }
            if (!role_wait(&accfull[buf], (it >> 1) & 1, P, et, eflag, 2, kEpi)) break;
            tc_fence_after();
            // Scatter of the upper triangle.  The atom images of a batch are ordered so that
            // every slot pair a <= b is the canonical member of its partner pair; element
            // (mu, nu) with mu <= nu therefore goes to block (a_mu, b_nu) at (o_mu, o_nu), and
            // the mirror kernel fills the other half.  Warp (q, hh) owns TMEM lanes 32q..32q+31
            // (orbitals row0..row0+31 of tile t) and the 32-column pieces c0 = 128 t + 32 hh + 64 k; a piece is
            // transposed through shared memory so that lanes = columns and the adds of a block
            // row are contiguous.  Addresses of 8 rows are formed before their atomics.
            float *tl = tiles + ew * 32 * 33;
            for (int t = 0; t < (nb > 128 ? 2 : 1); ++t) {
                const int row0 = t == 0 ? q * 32 : 128 + (q ^ 3) * 32;   // orbital of lane 0
                const int nrows = min(32, nb - row0);   // <= 0 for warps past the last row
                for (int c0 = t * 128 + hh * 32; c0 < npad; c0 += 64) {
                    if (nrows <= 0 || c0 + 32 <= row0) continue;   // wholly below the diagonal
                    float v[32];
                    const uint32_t col = (uint32_t)(base + t * npad + c0 - t * 128);
                    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + col;
                    tmem_ld16(taddr, v);
                    if (c0 + 16 < npad) tmem_ld16(taddr + 16, v + 16);
                    else
#pragma unroll
                        for (int j = 16; j < 32; ++j) v[j] = 0.f;
                    // the fp16 scaling is undone here for the row (this lane's TMEM lane) and in
                    // the scatter for the column (exact: powers of two)
                    float urow = 1.f, ucol = 1.f;
                    if constexpr (S::HALF) urow = pow2i(-eexp[min(row0 + lane, kMaxNb - 1)]);
#pragma unroll
                    for (int j = 0; j < 32; ++j) tl[j * 33 + lane] = v[j] * urow;
                    __syncwarp();
                    const int nu = c0 + lane;
                    const bool cv = nu < nb;
                    const int ci = info[cv ? nu : 0];
                    if constexpr (S::HALF) ucol = pow2i(-eexp[kMaxNb + (cv ? nu : 0)]);
                    const int b = ci & 255, ob = (ci >> 8) & 255, nbo = ci >> 16;
                    // rows in runs of one atom image (warp-uniform): one block lookup per run,
                    // then consecutive block rows are nbo doubles apart
                    for (int r = 0; r < nrows;) {
                        const int ri = info[row0 + r];
                        const int oa = (ri >> 8) & 255;
                        const int rend = min(nrows, r + (ri >> 16) - oa);
                        const int a = ri & 255;
                        const int e = small ? tbls[a * ns + b] : a <= b ? __ldg(tbl + tbl_index(a, b, ns)) : -1;
                        const bool blk = cv && e >= 0;
                        double *base = H + (e >> 1) + (oa - r) * nbo + ob;
                        const int rlim = min(rend, nu - row0 + 1);  // upper triangle: row <= nu
#pragma unroll 4
                        for (int r2 = r; r2 < rend; ++r2)
                            if (blk && r2 < rlim) red_add_f64(base + r2 * nbo, f2d_fast(tl[lane * 33 + r2] * ucol));
                        r = rend;
                    }
                    __syncwarp();
                }
            }
            tc_fence_before();
            mbar_arrive(&accempty[buf]);
            ++it;
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// ====================================================================== rho / force
// Psi_b = Phi_b D_b with M = 128 points and both N and K = the batch's orbitals in the padded
// layout (every slot rounded up to 8 columns, see kpad; slot s starts at koff[s]): Psi's TMEM
// columns and D's rows follow the same padded offsets.  The density matrix arrives pre-split: a
// per-call kernel writes its NT terms (scaled for fp16) into a padded store in which the units of
// one 16-byte block column (all rows, all terms) are adjacent, so the B operand of a chunk is
// assembled from bulk copies (one per core-matrix column and slot) with no arithmetic; the
// producers' only CUDA-core work is the orbital evaluation of the A operand.
//
// Operand layouts (K-major, no swizzle; core matrices of 8 rows x 16 bytes stored densely).
// A: the 8-row groups of one core-matrix column adjacent (SBO = 128 bytes) and the KCM columns
// of a chunk LBO = 128 x 16 bytes apart, so row r of column j sits at j * LBO + 16 r: producers
// with consecutive rows write consecutive 16 bytes.  B: per core-matrix column the 8-row groups
// of N in order, each with its NT terms side by side (SBO = NT x 128 bytes, term t at + 128 t).
constexpr int kRHalf = 256;          // producer warps 0-7 write the A operand
constexpr int kRBThr = 128;          // producer warps 8-11 copy the B operand
constexpr int kRProd = kRHalf + kRBThr;
constexpr int kRMma = kRProd;        // the MMA-issue thread (warp 12)
constexpr int kREpi0 = kRProd + 32;  // first epilogue thread (warp 13)
constexpr int kREPQ = 2;             // epilogue warps per TMEM lane quadrant
constexpr int kREpi = 128 * kREPQ;   // epilogue threads
constexpr int kThreadsR = kREpi0 + kREpi;

template <class S>
struct RL {
    static constexpr int CG = S::CG, NT = S::NT;
    static constexpr int KCM = 4;                      // core-matrix columns per chunk
    static constexpr int KC = KCM * CG;                // K columns per chunk (16 tf32, 32 16-bit)
    static constexpr int NS = NT == 2 ? 2 : 1;         // operand stages
    static constexpr int ESZ = 16 / CG;                // bytes per element
    static constexpr int LBO_A = kMaxBatchPts * 16;
    static constexpr int PLA = KCM * LBO_A;            // one A term of a chunk
    // B: [core-matrix column j][8-row group of N][term][row][16 bytes]: the terms of an 8-row
    // group adjacent (a term's 8-row groups SBO_B = NT x 128 bytes apart), columns LBO_B apart
    static constexpr int SBO_B = NT * 128;
    static constexpr int LBO_B = (kMaxNb / 8) * SBO_B;
    static constexpr int PLB = KCM * LBO_B;            // all B terms of a chunk
    // B, row layout (batches whose padded width exceeds the accumulator): term planes of PLBR
    // bytes, the N rows of a core-matrix column adjacent (SBO 128), columns LBO_BR apart
    static constexpr int LBO_BR = kMaxNb * 16;
    static constexpr int PLBR = KCM * LBO_BR;
    static_assert(NT * PLBR == PLB, "both B layouts fill the same stage");
    static constexpr int STAGE = NT * PLA + PLB;
    // producer metadata, double-buffered (the next batch's is copied during this one)
    static constexpr int OFF_PSLOT = NS * STAGE;                                    // PSlot[2][64]
    static constexpr int OFF_POFF = OFF_PSLOT + 2 * kMaxSlots * (int)sizeof(PSlot); // float [2][128][6]
    static constexpr int OFF_KOFF = OFF_POFF + 2 * kMaxBatchPts * 24;               // int [2][64]
    static constexpr int OFF_TBL = OFF_KOFF + 2 * kMaxSlots * 4;                    // int [2][kVTblR^2]
    static constexpr int OFF_KSLOT = OFF_TBL + 2 * kVTblR * kVTblR * 4;             // short [kMaxKCols / 8]
    static constexpr int OFF_KTASK = OFF_KSLOT + kMaxKCols / 8 * 2;                 // short [kMaxKCols / 8]
    static constexpr int OFF_EPSLOT = OFF_KTASK + kMaxKCols / 8 * 2;                // epilogue PSlot[64]
    static constexpr int OFF_EPOFF = OFF_EPSLOT + kMaxSlots * (int)sizeof(PSlot);
    static constexpr int OFF_WIN = OFF_EPOFF + kMaxBatchPts * 24;               // float [epilogue warps][32][32]
    static constexpr int OFF_RPART = OFF_WIN + (kREpi / 32) * 32 * 32 * 4;      // float [kREPQ][128]
    static constexpr int OFF_FACC = OFF_RPART + kREPQ * kMaxBatchPts * 4;       // float [64][3]
    static constexpr int OFF_BAR = (OFF_FACC + kMaxSlots * 12 + 15) / 16 * 16;  // 16 mbarriers
    static constexpr int OFF_MISC = OFF_BAR + 16 * 8;
    static constexpr int OFF_SPEC = OFF_MISC + 64;
    static constexpr int TOTAL = OFF_SPEC + kMaxSpecies * (int)sizeof(SpecSh);
};

// shared-memory descriptor with explicit strides (K-major, no swizzle)
__device__ __forceinline__ uint64_t sdesc2(uint32_t addr, uint32_t lbo, uint32_t sbo)
{
    return (uint64_t)((addr & 0x3FFFF) >> 4) | ((uint64_t)(lbo >> 4) << 16) | ((uint64_t)(sbo >> 4) << 32) |
           (1ull << 46);
}

// Split density-matrix store: every block (rows n_I, columns n_J, both padded to kpad with zeros)
// holds its NT terms at element NT soff[b] in 16-byte units of CG consecutive columns, ordered
// [column piece j][8-row group G][term t][row r]: unit (j, G, t, r) holds row 8 G + r, columns
// j CG .. j CG + CG - 1 of term t.  The units of one column piece (all rows, all terms) are
// adjacent, exactly as the B operand of the density kernel wants them in shared memory.
// sym: the block-symmetric part (DM + DM^T_block) / 2 (derivatives use it).  For fp16 the values
// are scaled by scale_for(max |DM|), read from amax.
//
// Row layout (padn == 0, decompositions whose padded width would exceed the accumulator): rows
// n_I, columns padded to kpad, term t in its own plane of `plane` elements; piece (i, c) (row i,
// columns c .. c + CG - 1) at soff[b] + (c / CG) n_I CG + i CG, so the rows of one piece are
// adjacent.
template <class S>
__global__ void k_dm_split(Plan P, const int *__restrict__ soff, const double *__restrict__ DM, void *out,
                           int64_t plane, int padn, int sym, const float *amax)
{
    constexpr int CG = S::CG, ESZ = 16 / CG, NT = S::NT;
    float sc = 1.f;
    if constexpr (S::HALF) sc = scale_for(amax[0]);
    unsigned char *o8 = reinterpret_cast<unsigned char *>(out);
    for (int64_t b = blockIdx.x; b < P.nblocks; b += gridDim.x) {
        const int64_t off = P.blk_off[b], poff = P.blk_off[P.partner[b]];
        const int rows = P.blk_rows[b];
        const int cols = (int)((P.blk_off[b + 1] - off) / rows);
        const int pr = padn ? kpad(rows) : rows, ng = pr / 8, npc = kpad(cols) / CG;
        unsigned char *base = o8 + (int64_t)(padn ? NT : 1) * soff[b] * ESZ;
        for (int e = threadIdx.x; e < pr * npc; e += blockDim.x) {
            const int j = e / pr, i = e - j * pr, c0 = j * CG;
            float x[CG];
#pragma unroll
            for (int q = 0; q < CG; ++q) {
                const int c = c0 + q;
                double v = 0.0;
                if (i < rows && c < cols)
                    v = sym ? 0.5 * (DM[off + i * cols + c] + DM[poff + c * rows + i]) : DM[off + i * cols + c];
                x[q] = d2f(v) * sc;
            }
            unsigned char *dst[NT];
#pragma unroll
            for (int t = 0; t < NT; ++t)
                dst[t] = padn ? base + (((j * ng + (i >> 3)) * NT + t) * 8 + (i & 7)) * 16
                              : base + ((int64_t)t * plane + (int64_t)c0 * rows + i * CG) * ESZ;
            split_store<S>(x, dst);
        }
    }
}

template <class S, bool RHO, bool FORCE, bool STRAIN>
__global__ void __launch_bounds__(kThreadsR, 1)
    k_rho_tc(Plan P, SInfo si0, const SInfo *__restrict__ sis)
{
    using L = RL<S>;
    constexpr int CG = L::CG, KCM = L::KCM, KC = L::KC, NS = L::NS, NT = S::NT;
    extern __shared__ __align__(1024) unsigned char sm[];
    PSlot *psb = reinterpret_cast<PSlot *>(sm + L::OFF_PSLOT);
    float *poffb = reinterpret_cast<float *>(sm + L::OFF_POFF);
    int *koffb = reinterpret_cast<int *>(sm + L::OFF_KOFF);
    int *tblb = reinterpret_cast<int *>(sm + L::OFF_TBL);
    short *kslot = reinterpret_cast<short *>(sm + L::OFF_KSLOT);
    short *ktask = reinterpret_cast<short *>(sm + L::OFF_KTASK);
    PSlot *eps = reinterpret_cast<PSlot *>(sm + L::OFF_EPSLOT);
    float *epoff = reinterpret_cast<float *>(sm + L::OFF_EPOFF);
    float *win = reinterpret_cast<float *>(sm + L::OFF_WIN);
    float *rpart = reinterpret_cast<float *>(sm + L::OFF_RPART);
    float *facc = reinterpret_cast<float *>(sm + L::OFF_FACC);
    SpecSh *spec = reinterpret_cast<SpecSh *>(sm + L::OFF_SPEC);
    uint64_t *bars = reinterpret_cast<uint64_t *>(sm + L::OFF_BAR);
    uint64_t *empty = bars, *accfull = bars + 2, *accempty = bars + 4, *fin = bars + 6, *full = bars + 8;
    uint64_t *bfull = bars + 10;   // the B operand's bulk copies of a stage have landed
    uint32_t *tmem_base = reinterpret_cast<uint32_t *>(sm + L::OFF_MISC);
    volatile int *pflag = reinterpret_cast<volatile int *>(sm + L::OFF_MISC + 4);
    volatile int *eflag = reinterpret_cast<volatile int *>(sm + L::OFF_MISC + 8);
    volatile int *bflag = reinterpret_cast<volatile int *>(sm + L::OFF_MISC + 12);

    const int tid = threadIdx.x, warp = tid >> 5;
    load_species(P, spec, tid);
    if (tid == 0) {
        mbar_init(&empty[0], 1);
        mbar_init(&empty[1], 1);
        mbar_init(&accfull[0], 1);
        mbar_init(&accfull[1], 1);
        mbar_init(&accempty[0], kREpi);
        mbar_init(&accempty[1], kREpi);
        mbar_init(fin, 1);
        mbar_init(&full[0], 2);   // one arrival from each producer group
        mbar_init(&full[1], 2);
        mbar_init(&bfull[0], 1);  // the B group's arrival and its copies' bytes
        mbar_init(&bfull[1], 1);
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

    if (tid < kRProd) {
        // ------------------------------------------------------------ producers
        const int pt = tid;
        int g = 0;
        int bph[2] = {0, 0};   // B group: phases of bfull[s] begun
        bool ok = true;
        SInfoCache sic(si0);
        CtaRange cr(P);
        int bi = 0, cur = 0;
        bool have = cr.next(bi);
        if (have)
            geom_async_rho(P, sis, si0, P.batches[bi], psb, poffb, koffb, tblb, pt, kRProd);
        for (; ok && have; have = cr.next(bi), cur ^= 1) {
            const Batch B = P.batches[bi];
            int n1, n2, n3;
            unpack(B.dims, n1, n2, n3);
            const int ns = B.nslots, nb = B.nb, npb = n1 * n2 * n3;
            const PSlot *ps = psb + cur * kMaxSlots;
            const float *poff = poffb + cur * kMaxBatchPts * 6;
            const int *koffs = koffb + cur * kMaxSlots;
            const int *tbls = tblb + cur * kVTblR * kVTblR;
            // this batch's metadata has arrived and every producer is done with the previous
            // batch (whose half of the buffers the next batch's copy overwrites)
            cp_async_wait_all();
            named_sync(4, kRProd);
            {
                CtaRange peek = cr;
                int bn = 0;
                if (peek.next(bn))
                    geom_async_rho(P, sis, si0, P.batches[bn], psb + (cur ^ 1) * kMaxSlots,
                                   poffb + (cur ^ 1) * kMaxBatchPts * 6, koffb + (cur ^ 1) * kMaxSlots,
                                   tblb + (cur ^ 1) * kVTblR * kVTblR, pt, kRProd);
            }
            if (nb == 0) continue;  // the epilogue writes rho = 0 there
            const SInfo SI = sic.get(B, sis);
            const bool tsm = ns <= kVTblR;
            const int ktot = (koffs[ns - 1] + kpad(ps[ns - 1].norb) + KC - 1) / KC * KC;
            // slot of each 8-column group of the padded K axis (-1: a gap): the last slot
            // starting at or before the group, if the group lies within its padded width.
            // ktask: the A task that starts at the group: -1 none (a gap), -2 the group is the
            // second half of a 16-column segment whose first half's task covers it, else the slot
            // | 128 when its values can stay in registers across the stage wait (a compiled
            // evaluator, its padded columns starting at the group and fitting the segment)
            for (int k8 = pt; k8 < ktot / 8; k8 += kRProd) {
                int lo = 0, hi = ns - 1;
                while (lo < hi) {
                    const int mid = (lo + hi + 1) >> 1;
                    if (koffs[mid] <= 8 * k8) lo = mid;
                    else hi = mid - 1;
                }
                const int ko = koffs[lo], kw = kpad(ps[lo].norb);
                const int sg = 8 * k8 < ko + kw ? lo : -1;
                kslot[k8] = (short)sg;
                int tk = sg;
                if (sg >= 0) {
                    if ((k8 & 1) && ko <= 8 * (k8 - 1)) tk = -2;
                    else if (spec[ps[sg].species].shape != kShapeGeneric && ko == 8 * k8 && kw <= 16 - 8 * (k8 & 1))
                        tk = sg | 128;
                }
                ktask[k8] = (short)tk;
            }
            named_sync(4, kRProd);
            float sA = 1.f;   // fp16: A = phi sA (the density matrix was scaled when it was split)
            if constexpr (S::HALF) sA = scale_for(SI.phimax);
            const unsigned char *dms = reinterpret_cast<const unsigned char *>(SI.DMS);
            const int nch = ktot / KC;
            // warps 0-7 write the A operand, warps 8-11 copy the B operand; each group waits for
            // the stage on its own and arrives on the stage's full barrier
            const bool agrp = pt < kRHalf;
            const int gt = agrp ? pt : pt - kRHalf;
            const int gbar = agrp ? 1 : 3, gthr = agrp ? kRHalf : kRBThr;
            volatile int *gflag = agrp ? pflag : bflag;
            const int p = gt % kMaxBatchPts;   // the A thread's point (the same in every unit)
            float po[6];
#pragma unroll
            for (int c = 0; c < 6; ++c) po[c] = poff[6 * (p < npb ? p : 0) + c];
            constexpr int NG = KC / 8;
            // A unit (thread, i): point p, 8-column group gq of the chunk.  Groups of the first
            // halves of 16-column segments come first; a thread's units lie in one segment.
            auto unit_group = [&](int i) {
                const int u = (gt + i * kRHalf) / kMaxBatchPts;
                return u < (NG + 1) / 2 ? 2 * u : 2 * (u - (NG + 1) / 2) + 1;
            };
            // A task classes (ktask): a register task keeps its values in registers across the
            // wait for the stage: xe for a task starting at the segment (first group), xo for one
            // starting at its second group.  Other tasks are evaluated after the wait.
            auto task_of = [&](int i, int k0, int &gq, int &sg, int &seg0, bool &reg) {
                gq = unit_group(i);
                const int v = ktask[(k0 >> 3) + gq];
                seg0 = k0 + (gq >> 1) * 16;
                reg = v >= 0 && (v & 128);
                sg = v < 0 ? v : (v & 127);
            };
            for (int ch = 0; ch < nch && ok; ++ch, ++g) {
                const int stage = g % NS;
                const int k0 = ch * KC;
                float xe[16], xo[8];
                if (agrp && p < npb) {
                    // A, first half (before the stage is free): register tasks evaluated
                    for (int i = 0; i * kRHalf + gt < NG * kMaxBatchPts; ++i) {
                        int gq, sg, seg0;
                        bool reg;
                        task_of(i, k0, gq, sg, seg0, reg);
                        if (!reg) continue;
                        const PSlot sl = ps[sg];
                        const SpecSh &sp = spec[sl.species];
                        float dx, dy, dz;
                        disp(sl, po, dx, dy, dz);
                        if (gq & 1) {
#pragma unroll
                            for (int q = 0; q < 8; ++q) xo[q] = 0.f;
                            if (sp.shape == kShapeSP) eval_phi_shape<ShapeSP>(sp, P.coef32, dx, dy, dz, [&](int o, float v) { xo[o] = v; }, sA);
                        } else {
#pragma unroll
                            for (int q = 0; q < 16; ++q) xe[q] = 0.f;
                            if (sp.shape == kShapeSPD) eval_phi_shape<ShapeSPD>(sp, P.coef32, dx, dy, dz, [&](int o, float v) { xe[o] = v; }, sA);
                            else eval_phi_shape<ShapeSP>(sp, P.coef32, dx, dy, dz, [&](int o, float v) { xe[o] = v; }, sA);
                        }
                    }
                }
                if (g >= NS) ok = role_wait(&empty[stage], ((g / NS) - 1) & 1, P, gt, gflag, gbar, gthr);
                if (!ok) break;
                unsigned char *st0 = sm + stage * L::STAGE;
                if (!agrp) {
                    // B: per (core-matrix column j of the chunk, slot b) the padded rows of slot b
                    // (N rows koff_b ..), all terms: in the split store these units of block (b, a)
                    // are adjacent, as they are in shared memory, so each is one bulk (TMA) copy
                    // of NT x 16 kpad(n_b) bytes that completes its bytes on bfull[stage]; zeros
                    // where the column is a gap or the pair has no block.  The copies bypass the
                    // load/store pipeline the orbital evaluations use.
                    uint32_t tx = 0;   // bytes of this thread's copies
                    if (!SI.padn) {
                        // row layout: per (term t, column j, slot b) the n_b rows, 16 n_b bytes
                        for (int w = (gt & 31) * (kRBThr / 32) + (gt >> 5); w < NT * KCM * ns; w += kRBThr) {
                            const int t = w / (KCM * ns), r = w - t * KCM * ns, j = r / ns, b = r - j * ns;
                            const int k = k0 + j * CG, a = kslot[k >> 3];
                            const int nbo = ps[b].norb;
                            unsigned char *dst = st0 + NT * L::PLA + t * L::PLBR + j * L::LBO_BR + ps[b].off * 16;
                            int e = -1;
                            if (a >= 0) e = tsm ? tbls[b * ns + a] : __ldg(P.tbl2 + B.tbl + b * ns + a);
                            if (e >= 0) {
                                const int64_t el = (int64_t)t * SI.dms_plane + e + ((k - koffs[a]) / CG) * nbo * CG;
                                bulk_g2s(dst, dms + el * L::ESZ, 16u * (uint32_t)nbo, &bfull[stage]);
                                tx += 16u * (uint32_t)nbo;
                            } else {
                                for (int row = 0; row < nbo; ++row)
                                    *reinterpret_cast<uint4 *>(dst + 16 * row) = make_uint4(0, 0, 0, 0);
                            }
                        }
                    }
                    // tasks dealt to the B warps in turn (a warp issues its bulk copies one lane
                    // after another, so the copies of a chunk are spread over all four warps)
                    const int bt = (gt & 31) * (kRBThr / 32) + (gt >> 5);
                    for (int w = bt; SI.padn && w < KCM * ns; w += kRBThr) {
                        const int j = w / ns, b = w - j * ns;
                        const int k = k0 + j * CG, a = kslot[k >> 3];
                        const int ng = kpad(ps[b].norb) / 8;
                        const uint32_t bytes = (uint32_t)(ng * L::SBO_B);
                        unsigned char *dst = st0 + NT * L::PLA + j * L::LBO_B + (koffs[b] / 8) * L::SBO_B;
                        int e = -1;
                        if (a >= 0) e = tsm ? tbls[b * ns + a] : __ldg(P.tbl2 + B.tbl + b * ns + a);
                        if (e >= 0) {
                            const int64_t unit = (int64_t)NT * e / CG + (int64_t)((k - koffs[a]) / CG) * ng * NT * 8;
                            bulk_g2s(dst, dms + unit * 16, bytes, &bfull[stage]);
                            tx += bytes;
                        } else {
                            for (uint32_t q = 0; q < bytes; q += 16)
                                *reinterpret_cast<uint4 *>(dst + q) = make_uint4(0, 0, 0, 0);
                        }
                    }
                    // one transaction count per warp (an expect before the copies' completions is
                    // not needed: the phase cannot complete before this group's arrival below)
                    tx = __reduce_add_sync(0xffffffffu, tx);
                    if ((gt & 31) == 0 && tx) mbar_expect_tx(&bfull[stage], tx);
                    ++bph[stage];
                } else {
                    // A, second half: each task's columns split into the operand row p (register
                    // tasks from their registers, the others evaluated now into a per-thread
                    // array); gaps zeroed.  Rows past the batch stay unwritten (their accumulator
                    // rows are not read).
                    for (int i = 0; i * kRHalf + gt < NG * kMaxBatchPts; ++i) {
                        int gq, sg, seg0;
                        bool reg;
                        task_of(i, k0, gq, sg, seg0, reg);
                        if (sg == -1) {
#pragma unroll
                            for (int t = 0; t < NT; ++t)
#pragma unroll
                                for (int q = 0; q < 8 / CG; ++q)
                                    *reinterpret_cast<uint4 *>(st0 + t * L::PLA + ((gq * 8) / CG + q) * L::LBO_A + p * 16) =
                                        make_uint4(0, 0, 0, 0);
                            continue;
                        }
                        if (sg < 0 || p >= npb) continue;
                        unsigned char *row = st0 + p * 16;
                        auto put = [&](int c, const float *x) {   // CG values (already scaled) of column c on
                            unsigned char *da[NT];
#pragma unroll
                            for (int t = 0; t < NT; ++t) da[t] = row + t * L::PLA + ((c - k0) / CG) * L::LBO_A;
                            split_store<S>(x, da);
                        };
                        if (reg) {
                            if (gq & 1) {
#pragma unroll
                                for (int c = 0; c < 8; c += CG) put(seg0 + 8 + c, xo + c);
                            } else {
                                const int kw = kpad(ps[sg].norb);
#pragma unroll
                                for (int c = 0; c < 16; c += CG)
                                    if (c < kw) put(seg0 + c, xe + c);
                            }
                            continue;
                        }
                        // other tasks: every orbital evaluated, the segment's columns kept
                        const PSlot sl = ps[sg];
                        const int ko = koffs[sg];
                        const int clo = max(ko, seg0), chi = min(ko + kpad(sl.norb), seg0 + 16);
                        float xl[16];
#pragma unroll
                        for (int q = 0; q < 16; ++q) xl[q] = 0.f;
                        float dx, dy, dz;
                        disp(sl, po, dx, dy, dz);
                        eval_phi_f32<false>(spec[sl.species], P.coef32, dx, dy, dz, [&](int o, float v) {
                            const int c = ko + o;
                            if (c >= clo && c < chi) xl[c - seg0] = v * sA;
                        });
                        for (int c = clo; c < chi; c += CG) put(c, xl + (c - seg0));
                    }
                }
                fence_async_smem();
                named_sync(gbar, gthr);
                if (gt == 0) {
                    mbar_arrive(&full[stage]);   // this group's half of chunk g is in place
                    // every B thread has registered its copies' bytes: the phase now completes
                    // when they have landed
                    if (!agrp) mbar_arrive(&bfull[stage]);
                }
            }
        }
        cp_async_wait_all();   // no copy may be in flight when the CTA exits
        if (pt == kRHalf) {
            // bulk copies of the last phase of each stage (consumed already unless a role gave up)
            for (int st = 0; st < NS; ++st)
                if (bph[st] > 0 && !mbar_wait(&bfull[st], (uint32_t)((bph[st] - 1) & 1), kDrainBudget)) report_timeout(P);
        }
    } else if (tid < kREpi0) {
        // ------------------------------------------------------------ MMA issue (one thread)
        if (tid == kRMma) {
            int g = 0, it = 0;
            bool ok = true;
            CtaRange cr(P);
            SInfoCache sic(si0);
            for (int bi = 0; ok && cr.next(bi);) {
                const Batch B = P.batches[bi];
                const int nb = B.nb;
                if (nb == 0) continue;
                const bool padn = sic.get(B, sis).padn != 0;
                const int buf = it & 1;
                const int last = B.slot0 + B.nslots - 1;
                const int kend = __ldg(P.koff + last) + kpad(P.tslots[last].norb);   // padded orbitals
                // N: the orbitals at their padded columns (padded layout) or unpadded
                const int npad = padn ? (kend + 15) & ~15 : (nb + 15) & ~15;
                const int ktot = (kend + KC - 1) / KC * KC;
                const int nch = ktot / KC;
                const uint32_t id = idesc<S>(128, npad);
                for (int ch = 0; ch < nch && ok; ++ch, ++g) {
                    const int stage = g % NS;
                    ok = !aborted(P) && mbar_wait(&full[stage], (g / NS) & 1, P.spin_limit) &&
                         mbar_wait(&bfull[stage], (g / NS) & 1, P.spin_limit);
                    if (ok && ch == 0 && it >= 2)   // the epilogue of batch it - 2 is done
                        ok = !aborted(P) && mbar_wait(&accempty[buf], ((it >> 1) - 1) & 1, P.spin_limit);
                    if (!ok) {
                        report_timeout(P);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = su32(sm + stage * L::STAGE), b0 = a0 + NT * L::PLA;
#pragma unroll
                    for (int ks = 0; ks < KCM / 2; ++ks) {
#pragma unroll
                        for (int q = 0; q < S::NPROD; ++q) {
                            const uint64_t da = sdesc2(a0 + term(S::PA, q) * L::PLA + ks * 2 * L::LBO_A, L::LBO_A, 128);
                            const uint64_t db =
                                padn ? sdesc2(b0 + term(S::PB, q) * 128 + ks * 2 * L::LBO_B, L::LBO_B, L::SBO_B)
                                     : sdesc2(b0 + term(S::PB, q) * L::PLBR + ks * 2 * L::LBO_BR, L::LBO_BR, 128);
                            const uint32_t acc = (ch == 0 && ks == 0 && q == 0) ? 0u : 1u;
                            umma<S::F16>(tmem + buf * 256, da, db, id, acc);
                        }
                    }
                    umma_commit(&empty[stage]);
                    if (ch == nch - 1) umma_commit(&accfull[buf]);
                }
                ++it;
            }
            umma_commit(fin);
            if (!mbar_wait(fin, 0, kDrainBudget)) report_timeout(P);
        }
    } else {
        // ------------------------------------------------------------ epilogue: rho and force
        // warp (q, hh): TMEM lane quadrant q = warp % 4 (points 32q..32q+31), the hh-th of the
        // quadrant's kREPQ warps
        const int et = tid - kREpi0, ew = et >> 5, lane = et & 31;
        const int q = warp & 3, hh = ew >> 2;
        const int p = q * 32 + lane;  // TMEM lane = point of the batch
        float *w = win + ew * 32 * 32;
        int it = 0;
        // strain derivative (single-structure launches): [0..8] Sum V grad_a phi . Psi d_b,
        // [9] Sum V rho, over this thread's points and atom images
        const bool strain = STRAIN && FORCE && si0.dLde != nullptr && sis == nullptr;
        double sacc[10];
#pragma unroll
        for (int k = 0; k < 10; ++k) sacc[k] = 0.0;
        SInfoCache sic(si0);
        CtaRange cr(P);
        for (int bi = 0; cr.next(bi);) {
            const Batch B = P.batches[bi];
            int n1, n2, n3;
            unpack(B.dims, n1, n2, n3);
            const int ns = B.nslots, npb = n1 * n2 * n3;
            const int buf = it & 1;
            const SInfo SI = sic.get(B, sis);
            if (B.nb == 0) {
                if (RHO && hh == 0 && p < npb) SI.rho[grid_index(SI, B, p, n2, n3)] = 0.0;
                continue;
            }
            named_sync(2, kREpi);
            load_geom(P, SI, B, eps, epoff, et, kREpi);
            if (SI.padn)
                for (int s = et; s < ns; s += kREpi) eps[s].off = __ldg(P.koff + B.slot0 + s);   // padded N column
            if (FORCE)
                for (int e = et; e < 3 * ns; e += kREpi) facc[e] = 0.f;
            if (!role_wait(&accfull[buf], (it >> 1) & 1, P, et, eflag, 2, kREpi)) break;
            tc_fence_after();
            const bool pv = p < npb;
            const uint32_t trow = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * 256);
            float vp = 0.f;
            int64_t gi = 0;
            float u = 1.f;   // undoes the fp16 operand scaling of Psi (exact: a power of two)
            if constexpr (S::HALF) u = 1.f / (scale_for(SI.phimax) * scale_for(SI.amax[1]));
            if (pv) {
                gi = grid_index(SI, B, p, n2, n3);
                if (FORCE) vp = d2f(SI.V[gi]);
            }
            const float vpu = vp * u;
            float po[6];   // this point's offset from the batch origin (hi, lo)
#pragma unroll
            for (int c = 0; c < 6; ++c) po[c] = epoff[6 * (pv ? p : 0) + c];
            float racc = 0.f;
            float st[9];
#pragma unroll
            for (int k = 0; k < 9; ++k) st[k] = 0.f;
            // this warp's atom images: a contiguous range; two consecutive images of one species
            // whose columns fit one 32-column window are evaluated together (two independent
            // chains for the scheduler), the others one by one
            auto slot_done = [&](int s, float fx, float fy, float fz, float dx, float dy, float dz) {
                if (strain) {
                    st[0] += fx * dx; st[1] += fx * dy; st[2] += fx * dz;
                    st[3] += fy * dx; st[4] += fy * dy; st[5] += fy * dz;
                    st[6] += fz * dx; st[7] += fz * dy; st[8] += fz * dz;
                }
                if (FORCE && SI.F) {
                    fx *= vpu; fy *= vpu; fz *= vpu;
#pragma unroll
                    for (int m = 16; m > 0; m >>= 1) {
                        fx += __shfl_xor_sync(0xffffffffu, fx, m);
                        fy += __shfl_xor_sync(0xffffffffu, fy, m);
                        fz += __shfl_xor_sync(0xffffffffu, fz, m);
                    }
                    if (lane == 0) {
                        // the four lane quadrants of a slot meet here: FP32 shared-memory adds,
                        // FP64 from the per-batch sum on
                        atomicAdd(&facc[3 * s + 0], fx);
                        atomicAdd(&facc[3 * s + 1], fy);
                        atomicAdd(&facc[3 * s + 2], fz);
                    }
                }
            };
            auto load_window = [&](int w0, int wn) {
                for (int c = 0; c < wn; c += 16) {
                    uint32_t v[16];
                    tmem_ld16_async(trow + (uint32_t)(w0 + c), v);
                    tmem_wait_ld();
#pragma unroll
                    for (int j = 0; j < 16; ++j) w[(c + j) * 32 + lane] = __uint_as_float(v[j]);
                }
                __syncwarp();
            };
            const int s_end = (ns * (hh + 1)) / kREPQ;
            for (int s = (ns * hh) / kREPQ; s < s_end;) {
                const PSlot sa = eps[s];
                const int w0 = sa.off & ~15;
                const bool pair = s + 1 < s_end && eps[s + 1].species == sa.species &&
                                  eps[s + 1].off + eps[s + 1].norb <= w0 + 32 && spec[sa.species].shape != kShapeGeneric;
                if (pair) {
                    const PSlot sb = eps[s + 1];
                    const SpecSh &sp = spec[sa.species];
                    float ax = 0.f, ay = 0.f, az = 0.f, bx = 0.f, by = 0.f, bz = 0.f;
                    if (pv) {
                        disp(sa, po, ax, ay, az);
                        disp(sb, po, bx, by, bz);
                    }
                    const bool ina = pv && ax * ax + ay * ay + az * az < sp.rcut2;
                    const bool inb = pv && bx * bx + by * by + bz * bz < sp.rcut2;
                    load_window(w0, ((sb.off + sb.norb - w0) + 15) & ~15);
                    float fax = 0.f, fay = 0.f, faz = 0.f, fbx = 0.f, fby = 0.f, fbz = 0.f;
                    if (__any_sync(0xffffffffu, ina || inb)) {
                        // both images evaluated unconditionally (finite outside the sphere: the
                        // interval index is clamped) and masked, so the two chains interleave;
                        // displacements below 1e-12 take the generic centre limits
                        const int ca = sa.off - w0, cb2 = sb.off - w0;
                        float ra = 0.f, rb = 0.f;
                        const float a2 = ina ? ax : 1.f, ay2 = ina ? ay : 0.f, az2 = ina ? az : 0.f;
                        const float b2 = inb ? bx : 1.f, by2 = inb ? by : 0.f, bz2 = inb ? bz : 0.f;
                        eval_rho_grad_any<FORCE>(sp, P.coef32, a2, ay2, az2, [&](int o) { return w[(ca + o) * 32 + lane]; },
                                                 ra, fax, fay, faz);
                        eval_rho_grad_any<FORCE>(sp, P.coef32, b2, by2, bz2, [&](int o) { return w[(cb2 + o) * 32 + lane]; },
                                                 rb, fbx, fby, fbz);
                        if (!ina) ra = fax = fay = faz = 0.f;
                        if (!inb) rb = fbx = fby = fbz = 0.f;
                        racc += ra + rb;
                    }
                    __syncwarp();
                    slot_done(s, fax, fay, faz, ax, ay, az);
                    slot_done(s + 1, fbx, fby, fbz, bx, by, bz);
                    s += 2;
                    continue;
                }
                float fx = 0.f, fy = 0.f, fz = 0.f;
                float dx = 0.f, dy = 0.f, dz = 0.f;
                if (pv) disp(sa, po, dx, dy, dz);
                // a point outside the image's sphere adds nothing (the window loads stay
                // warp-uniform)
                const bool in = pv && dx * dx + dy * dy + dz * dz < spec[sa.species].rcut2;
                // orbitals [oa, ob) of the slot whose columns fit one 32-column window (all of
                // them unless the slot has more than 17 orbitals)
                for (int oa = 0; oa < sa.norb;) {
                    const int ob = min(sa.norb, ((sa.off + oa) & ~15) + 32 - sa.off);
                    const int v0 = (sa.off + oa) & ~15;
                    load_window(v0, ((sa.off + ob - v0) + 15) & ~15);
                    const int cb = sa.off - v0;   // window column of orbital o: cb + o
                    if (in)
                        eval_rho_grad_any<FORCE>(
                            spec[sa.species], P.coef32, dx, dy, dz,
                            [&](int o) { return (o >= oa && o < ob) ? w[(cb + o) * 32 + lane] : 0.f; }, racc, fx, fy,
                            fz);
                    __syncwarp();
                    oa = ob;
                }
                slot_done(s, fx, fy, fz, dx, dy, dz);
                ++s;
            }
            tc_fence_before();
            mbar_arrive(&accempty[buf]);
            racc *= u;
            if (RHO) rpart[hh * kMaxBatchPts + p] = racc;
            named_sync(2, kREpi);
            if (RHO && hh == 0 && pv) {
                float rs = 0.f;
#pragma unroll
                for (int k = 0; k < kREPQ; ++k) rs += rpart[k * kMaxBatchPts + p];
                SI.rho[gi] = f2d(rs);
            }
            if (FORCE && SI.F)
                for (int e = et; e < 3 * ns; e += kREpi)
                    red_add_f64(&SI.F[3 * eps[e / 3].atom + e % 3], 2.0 * SI.dV * f2d(facc[e]));
            if (strain && pv) {
#pragma unroll
                for (int k = 0; k < 9; ++k) sacc[k] += f2d(vpu * st[k]);
                sacc[9] += f2d(vp * racc);
            }
            ++it;
        }
        if (strain) {
            // dL/deps_ab = 2 dV Sum V grad_a phi . Psi d_b + delta_ab dV Sum V rho
#pragma unroll
            for (int k = 0; k < 10; ++k)
#pragma unroll
                for (int m = 16; m > 0; m >>= 1) sacc[k] += __shfl_xor_sync(0xffffffffu, sacc[k], m);
            if (lane == 0)
                for (int k = 0; k < 9; ++k)
                    red_add_f64(&si0.dLde[k], 2.0 * si0.dV * sacc[k] + ((k % 4) == 0 ? si0.dV * sacc[9] : 0.0));
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols));
    }
}

// Ask for the smallest shared-memory carveout that holds `smem` bytes, so the rest of the
// unified L1/shared storage caches the spline records.
template <class K>
cudaError_t set_smem(K kernel, int smem)
{
    cudaError_t e = cudaFuncSetAttribute(kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
    if (e != cudaSuccess) return e;
    static const int cfg[] = {0, 8, 16, 32, 64, 100, 132, 164, 196, 228};   // KiB
    const int need = (smem + 1024 + 1023) / 1024;                         // + the driver's 1 KiB
    int kib = 228;
    for (int c : cfg)
        if (c >= need) {
            kib = c;
            break;
        }
    return cudaFuncSetAttribute(kernel, cudaFuncAttributePreferredSharedMemoryCarveout, kib * 100 / 228);
}

template <class S>
cudaError_t vlocal_launch(const Plan &P, const SInfo &si0, const SInfo *sis, cudaStream_t s, int nsm, int max_nb)
{
    constexpr int smem = VSmem<S>::TOTAL;
    static_assert(smem <= 232448, "vlocal shared memory");
    cudaError_t e = set_smem(k_vlocal_tc<S>, smem);
    if (e != cudaSuccess) return e;
    const int grid = P.rng ? P.npart : std::min(nsm, P.nbatches);
    (void)max_nb;
    k_vlocal_tc<S><<<grid, kThreadsTC, smem, s>>>(P, si0, sis);
    return cudaGetLastError();
}

template <class S, bool R, bool Fo, bool St>
cudaError_t rho_launch3(const Plan &P, const SInfo &si0, const SInfo *sis, cudaStream_t s, int nsm)
{
    constexpr int smem = RL<S>::TOTAL;
    static_assert(smem <= 232448, "rho shared memory");
    cudaError_t e = set_smem(k_rho_tc<S, R, Fo, St>, smem);
    if (e != cudaSuccess) return e;
    const int grid = P.rng ? P.npart : std::min(nsm, P.nbatches);
    k_rho_tc<S, R, Fo, St><<<grid, kThreadsR, smem, s>>>(P, si0, sis);
    return cudaGetLastError();
}

template <class S>
cudaError_t dm_split_launch(const Plan &P, const int *soff, const double *DM, void *out, int64_t plane, bool padn,
                            bool sym, const float *amax, cudaStream_t s)
{
    const int grid = (int)std::min<int64_t>(P.nblocks, 8192);
    if (grid < 1) return cudaSuccess;
    k_dm_split<S><<<grid, 128, 0, s>>>(P, soff, DM, out, plane, padn ? 1 : 0, sym ? 1 : 0, amax);
    return cudaGetLastError();
}

template <class S>
cudaError_t rho_launch(const Plan &P, const SInfo &si0, const SInfo *sis, bool rho, bool force, cudaStream_t s,
                       int nsm)
{
    // the strain derivative has its own instantiation, so the other paths keep its
    // accumulators out of their registers
    if (si0.dLde) return rho_launch3<S, false, true, true>(P, si0, sis, s, nsm);
    if (rho && force) return rho_launch3<S, true, true, false>(P, si0, sis, s, nsm);
    if (rho) return rho_launch3<S, true, false, false>(P, si0, sis, s, nsm);
    return rho_launch3<S, false, true, false>(P, si0, sis, s, nsm);
}

}  // namespace

cudaError_t launch_vlocal_tc(const Plan &P, gint_prec prec, const SInfo &si0, const SInfo *sis, cudaStream_t s,
                             int nsm, int max_nb)
{
    if (P.nbatches == 0) return cudaSuccess;
    switch (prec) {
    case GINT_TF32X3: return vlocal_launch<TF32x3W>(P, si0, sis, s, nsm, max_nb);
    case GINT_BF16X3: return vlocal_launch<BF16x3W>(P, si0, sis, s, nsm, max_nb);
    case GINT_BF16X6: return vlocal_launch<BF16x6W>(P, si0, sis, s, nsm, max_nb);
    case GINT_FP16X3: return vlocal_launch<FP16x3W>(P, si0, sis, s, nsm, max_nb);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_dm_split(const Plan &P, gint_prec prec, const int *soff, const double *DM, void *out,
                            int64_t plane, bool padn, bool sym, const float *amax, cudaStream_t s)
{
    switch (prec) {
    case GINT_TF32X3: return dm_split_launch<TF32x3W>(P, soff, DM, out, plane, padn, sym, amax, s);
    case GINT_BF16X3: return dm_split_launch<BF16x3W>(P, soff, DM, out, plane, padn, sym, amax, s);
    case GINT_BF16X6: return dm_split_launch<BF16x6W>(P, soff, DM, out, plane, padn, sym, amax, s);
    case GINT_FP16X3: return dm_split_launch<FP16x3W>(P, soff, DM, out, plane, padn, sym, amax, s);
    default: return cudaErrorInvalidValue;
    }
}

cudaError_t launch_rho_force_tc(const Plan &P, gint_prec prec, const SInfo &si0, const SInfo *sis, bool rho,
                                bool force, cudaStream_t s, int nsm)
{
    if (P.nbatches == 0) return cudaSuccess;
    switch (prec) {
    case GINT_TF32X3: return rho_launch<TF32x3W>(P, si0, sis, rho, force, s, nsm);
    case GINT_BF16X3: return rho_launch<BF16x3W>(P, si0, sis, rho, force, s, nsm);
    case GINT_BF16X6: return rho_launch<BF16x6W>(P, si0, sis, rho, force, s, nsm);
    case GINT_FP16X3: return rho_launch<FP16x3W>(P, si0, sis, rho, force, s, nsm);
    default: return cudaErrorInvalidValue;
    }
}

}  // namespace gint
