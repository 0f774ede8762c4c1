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

// ------------------------------------------------------------------ shared batch metadata
// An atom image of the batch in shared memory: the first 16 bytes and dh/dl as in Slot, so
// they can be copied asynchronously in 8-byte pieces.
struct PSlot {
    int atom, species, off, norb;
    float dh[3], dl[3];
};
static_assert(sizeof(PSlot) == 40, "PSlot layout");
static_assert(offsetof(Slot, dh) == 40 && sizeof(Slot) == 64, "Slot layout");

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
        const Slot &S = P.slots[B.slot0 + s];
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
        const char *src = reinterpret_cast<const char *>(P.slots + B.slot0 + s);
        char *dst = reinterpret_cast<char *>(ps + s);
        if (part < 2) cp_async8(dst + 8 * part, src + 8 * part);           // atom .. norb
        else cp_async8(dst + 8 * part, src + 24 + 8 * part);               // dh, dl
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

__device__ __forceinline__ void disp(const PSlot &s, const float *po, float &dx, float &dy, float &dz)
{
    dx = (s.dh[0] + po[0]) + (s.dl[0] + po[3]);
    dy = (s.dh[1] + po[1]) + (s.dl[1] + po[4]);
    dz = (s.dh[2] + po[2]) + (s.dl[2] + po[5]);
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
        spec[tid] = q;
    }
}

// ====================================================================== vlocal
// With nbuf = 2 (every batch <= 192 orbitals) TMEM accumulator buffer b occupies columns
// [256 b, 256 b + 256): tile 0 (rows 0..127, N = npad <= 192) at +0 and tile 1 (rows 128..,
// N = npad - 128 <= 64) at +192.  With nbuf = 1 (some batch has up to 256 orbitals) one
// accumulator holds tile 0 at columns [0, 256) and tile 1 at [256, 384).
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
    static constexpr int OFF_VD = OFF_POFF + 2 * kMaxBatchPts * 6 * 4;      // double [2][128]
    static constexpr int OFF_V = OFF_VD + 2 * kMaxBatchPts * 8;             // float [128]
    static constexpr int OFF_TBL = OFF_V + kMaxBatchPts * 4;                // int [kVTbl^2]
    static constexpr int OFF_INFO = OFF_TBL + kVTbl * kVTbl * 4;            // int [256]: slot | o << 8 | norb << 16
    static constexpr int OFF_TILE = OFF_INFO + kMaxNb * 4;                  // float [8][32][33]
    static constexpr int OFF_BAR = OFF_TILE + 8 * 32 * 33 * 4;              // 16 mbarriers
    static constexpr int OFF_MISC = OFF_BAR + 16 * 8;                       // tmem base, flags
    static constexpr int OFF_SPEC = OFF_MISC + 64;                          // SpecSh[kMaxSpecies]
    static constexpr int TOTAL = OFF_SPEC + kMaxSpecies * (int)sizeof(SpecSh);
};

template <class S>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_vlocal_tc(Plan P, SInfo si0, const SInfo *__restrict__ sis, int nbuf)
{
    using L = VSmem<S>;
    constexpr int KC = L::KC, NS = L::NSTAGE;
    constexpr int SBO = S::KCM * kLBO;
    extern __shared__ __align__(1024) unsigned char sm[];
    float *stg = reinterpret_cast<float *>(sm + L::OFF_STG);
    PSlot *psb = reinterpret_cast<PSlot *>(sm + L::OFF_PSLOT);
    float *poffb = reinterpret_cast<float *>(sm + L::OFF_POFF);
    double *vdb = reinterpret_cast<double *>(sm + L::OFF_VD);
    float *vs = reinterpret_cast<float *>(sm + L::OFF_V);
    int *tbls = reinterpret_cast<int *>(sm + L::OFF_TBL);
    int *info = reinterpret_cast<int *>(sm + L::OFF_INFO);
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
    const int tile1 = nbuf == 2 ? 192 : 256;   // TMEM column of tile 1 within an accumulator

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
        if (have) geom_async(P, sis, si0, P.batches[bi], psb, poffb, vdb, pt, kProd);
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
                                     vdb + (cur ^ 1) * kMaxBatchPts, pt, kProd);
                continue;
            }
            const SInfo SI = sic.get(B, sis);
            float dVf = (float)SI.dV, sA = 1.f;
            if constexpr (S::HALF) {
                // fp16 operands: A = phi sA, B = V dV phi sB (powers of two, undone in the epilogue)
                sA = scale_for(SI.phimax);
                dVf *= scale_for(SI.amax[0] * dVf * SI.phimax);
            }
            for (int p = pt; p < kMaxBatchPts; p += kProd)
                vs[p] = p < npb ? d2f(vdb[cur * kMaxBatchPts + p]) * dVf : 0.f;
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
                        eval_phi_f32<!S::F16>(spec[sl.species], P.coef32, dx, dy, dz, [&](int o, float v) { col[o * KC] = v; });
                    } else {
                        for (int o = 0; o < sl.norb; ++o) col[o * KC] = 0.f;
                    }
                }
                if (ch == 0 && more)
                    geom_async(P, sis, si0, Bn, psb + (cur ^ 1) * kMaxSlots, poffb + (cur ^ 1) * kMaxBatchPts * 6,
                               vdb + (cur ^ 1) * kMaxBatchPts, pt, kProd);
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
#pragma unroll
                        for (int i = 0; i < S::CG; ++i) {
                            x[i] = stg[row * KC + kc * S::CG + i];
                            y[i] = x[i] * vs[ch * KC + kc * S::CG + i];
                            if constexpr (S::HALF) x[i] *= sA;
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
            for (int bi = 0; ok && cr.next(bi);) {
                const Batch B = P.batches[bi];
                int n1, n2, n3;
                unpack(B.dims, n1, n2, n3);
                const int nb = B.nb, npb = n1 * n2 * n3;
                if (nb == 0) continue;
                const int npad = (nb + 15) & ~15;
                const int buf = nbuf == 2 ? (it & 1) : 0;
                const int nch = (npb + KC - 1) / KC;
                for (int ch = 0; ch < nch && ok; ++ch, ++g) {
                    const int stage = g % NS;
                    ok = !aborted(P) && mbar_wait(&full[stage], (g / NS) & 1, P.spin_limit);
                    if (ok && ch == 0 && it >= nbuf)   // the epilogue of batch it - nbuf is done
                        ok = !aborted(P) && mbar_wait(&accempty[buf], ((it / nbuf) - 1) & 1, P.spin_limit);
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
                                umma<S::F16>(tmem + buf * 256 + t * tile1, da, db, id, acc);
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
        for (int bi = 0; cr.next(bi);) {
            const Batch B = P.batches[bi];
            const int ns = B.nslots, nb = B.nb;
            const int npad = (nb + 15) & ~15;
            const int buf = nbuf == 2 ? (it & 1) : 0;
            if (nb == 0) continue;
            const SInfo SIe = sic.get(B, sis);
            double *H = SIe.H;
            float u = 1.f;   // undoes the fp16 operand scaling (exact: a power of two)
            if constexpr (S::HALF) {
                const float dVf = (float)SIe.dV;
                u = 1.f / (scale_for(SIe.phimax) * scale_for(SIe.amax[0] * dVf * SIe.phimax));
            }
            const bool small = ns <= kVTbl;
            const int *tbl = small ? tbls : P.tbl + B.tbl;
            named_sync(2, kEpi);
            if (small)
                for (int e = et; e < ns * ns; e += kEpi) tbls[e] = P.tbl[B.tbl + e];
            for (int s = et; s < ns; s += kEpi) {
                const Slot &sl = P.slots[B.slot0 + s];
                const int no = sl.norb, off = sl.orb_off;
                for (int o = 0; o < no; ++o) info[off + o] = s | (o << 8) | (no << 16);
            }
            if (!role_wait(&accfull[buf], (it / nbuf) & 1, P, et, eflag, 2, kEpi)) break;
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
                    const uint32_t col = (uint32_t)(buf * 256 + t * tile1 + c0 - t * 128);
                    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + col;
                    tmem_ld16(taddr, v);
                    if (c0 + 16 < npad) tmem_ld16(taddr + 16, v + 16);
                    else
#pragma unroll
                        for (int j = 16; j < 32; ++j) v[j] = 0.f;
#pragma unroll
                    for (int j = 0; j < 32; ++j) tl[j * 33 + lane] = v[j];
                    __syncwarp();
                    const int nu = c0 + lane;
                    const bool cv = nu < nb;
                    const int ci = info[cv ? nu : 0];
                    const int b = ci & 255, ob = (ci >> 8) & 255, nbo = ci >> 16;
                    // rows in runs of one atom image (warp-uniform): one block lookup per run,
                    // then consecutive block rows are nbo doubles apart
                    for (int r = 0; r < nrows;) {
                        const int ri = info[row0 + r];
                        const int oa = (ri >> 8) & 255;
                        const int rend = min(nrows, r + (ri >> 16) - oa);
                        const int e = tbl[(ri & 255) * ns + b];
                        const bool blk = cv && e >= 0;
                        double *base = H + (e >> 1) + (oa - r) * nbo + ob;
                        const int rlim = min(rend, nu - row0 + 1);  // upper triangle: row <= nu
#pragma unroll 4
                        for (int r2 = r; r2 < rend; ++r2)
                            if (blk && r2 < rlim) red_add_f64(base + r2 * nbo, f2d_fast(tl[lane * 33 + r2] * u));
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
template <class S>
struct RSmem {
    static constexpr int KC = S::KCM * S::CG;              // orbitals per chunk
    static constexpr int RING = 64;                        // staging rows (orbital ring, see k_rho_tc)
    static constexpr int EG = KC >= 32 ? 1 : 32 / KC;      // chunks per orbital evaluation
    static constexpr int ARR_A = arr_bytes<S>(kMaxBatchPts);
    static constexpr int ARR_B = arr_bytes<S>(kMaxNb);
    static constexpr int STAGE = S::NT * (ARR_A + ARR_B);
    // stages per scheme: with one, the MMAs of a chunk overlap the next chunk's orbital
    // evaluation and gather tables, which come before the stage is rewritten
    static constexpr int NSTAGE = S::RSTAGES;
    static constexpr int OFF_STG = NSTAGE * STAGE;                          // float [RING][128]
    static constexpr int OFF_PSLOT = OFF_STG + RING * kMaxBatchPts * 4;     // producer PSlot[64]
    static constexpr int OFF_POFF = OFF_PSLOT + kMaxSlots * (int)sizeof(PSlot);
    static constexpr int OFF_OMAP = OFF_POFF + kMaxBatchPts * 24;           // oslot[256], oidx[256]
    static constexpr int OFF_GBASE = OFF_OMAP + 2 * kMaxNb;                 // int [64][KC]: chunk gather bases
    static constexpr int OFF_GNA = OFF_GBASE + kMaxSlots * KC * 4;          // int [KC]: norb of column's slot
    static constexpr int OFF_EPSLOT = OFF_GNA + KC * 4;                     // epilogue PSlot[64]
    static constexpr int OFF_EPOFF = OFF_EPSLOT + kMaxSlots * (int)sizeof(PSlot);
    static constexpr int OFF_WIN = OFF_EPOFF + kMaxBatchPts * 24;           // float [8][kWin][32]
    static constexpr int OFF_RPART = OFF_WIN + 8 * kWin * 32 * 4;           // float [128]
    static constexpr int OFF_FACC = OFF_RPART + kMaxBatchPts * 4;           // float [64][3]
    static constexpr int OFF_BAR = OFF_FACC + kMaxSlots * 3 * 4;             // 16 mbarriers
    static constexpr int OFF_MISC = OFF_BAR + 16 * 8;
    static constexpr int OFF_SPEC = OFF_MISC + 64;
    static constexpr int TOTAL = OFF_SPEC + kMaxSpecies * (int)sizeof(SpecSh);
};

template <class S, bool RHO, bool FORCE, bool STRAIN>
__global__ void __launch_bounds__(kThreadsTC, 1)
    k_rho_tc(Plan P, SInfo si0, const SInfo *__restrict__ sis)
{
    using L = RSmem<S>;
    constexpr int KC = L::KC, RING = L::RING, EG = L::EG, NS = L::NSTAGE;
    constexpr int SBO = S::KCM * kLBO;
    extern __shared__ __align__(1024) unsigned char sm[];
    float *stg = reinterpret_cast<float *>(sm + L::OFF_STG);
    PSlot *ps = reinterpret_cast<PSlot *>(sm + L::OFF_PSLOT);
    float *poff = reinterpret_cast<float *>(sm + L::OFF_POFF);
    unsigned char *oslot = sm + L::OFF_OMAP, *oidx = oslot + kMaxNb;
    int *gbase = reinterpret_cast<int *>(sm + L::OFF_GBASE);
    int *gna = reinterpret_cast<int *>(sm + L::OFF_GNA);
    // slot-pair table of a batch with at most kVTbl atom images, in the tail of the gather
    // bases (which then use at most kVTbl * KC entries)
    static_assert(kVTbl * KC + kVTbl * kVTbl <= kMaxSlots * KC, "slot-pair table placement");
    int *rtbl = gbase + kMaxSlots * KC - kVTbl * kVTbl;
    PSlot *eps = reinterpret_cast<PSlot *>(sm + L::OFF_EPSLOT);
    float *epoff = reinterpret_cast<float *>(sm + L::OFF_EPOFF);
    float *win = reinterpret_cast<float *>(sm + L::OFF_WIN);
    float *rpart = reinterpret_cast<float *>(sm + L::OFF_RPART);
    SpecSh *spec = reinterpret_cast<SpecSh *>(sm + L::OFF_SPEC);
    float *facc = reinterpret_cast<float *>(sm + L::OFF_FACC);
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
        // ------------------------------------------------------------ producers + MMA issue
        const int pt = tid;
        int g = 0;
        bool ok = true;
        // Orbital ring: when every slot fits (EG KC + norb - 1 <= RING rows), the orbitals of a
        // slot are evaluated once, every EG chunks for the slots that start in those chunks, into
        // staging rows (orbital index) mod RING; later chunks read the rows carried over.
        // Otherwise each chunk evaluates every slot overlapping it and keeps its own columns.
        int maxnorb = 0;
        for (int i = 0; i < P.nspecies; ++i) maxnorb = max(maxnorb, P.sp[i].norb);
        const bool ring = EG * KC + maxnorb - 1 <= RING;
        SInfoCache sic(si0);
        CtaRange cr(P);
        for (int bi = 0; ok && cr.next(bi);) {
            const Batch B = P.batches[bi];
            int n1, n2, n3;
            unpack(B.dims, n1, n2, n3);
            const int ns = B.nslots, nb = B.nb, npb = n1 * n2 * n3;
            const int npad = (nb + 15) & ~15;
            if (nb == 0) continue;  // the epilogue writes rho = 0 there
            const SInfo SI = sic.get(B, sis);
            const float *__restrict__ DM = SI.DM32;
            const int *__restrict__ tbl = P.tbl + B.tbl;
            float sA = 1.f, sD = 1.f;   // fp16 operands: A = phi sA, B = D sD (undone in the epilogue)
            if constexpr (S::HALF) {
                sA = scale_for(SI.phimax);
                sD = scale_for(SI.amax[1]);
            }
            named_sync(1, kProd);
            load_geom(P, SI, B, ps, poff, pt, kProd);
            // the batch's slot-pair table in shared memory (gather tables read it per chunk)
            const bool tsm = ns <= kVTbl;
            if (tsm)
                for (int e = pt; e < ns * ns; e += kProd) rtbl[e] = __ldg(tbl + e);
            named_sync(1, kProd);
            for (int s = pt; s < ns; s += kProd)
                for (int o = 0; o < ps[s].norb; ++o) {
                    oslot[ps[s].off + o] = (unsigned char)s;
                    oidx[ps[s].off + o] = (unsigned char)o;
                }
            named_sync(1, kProd);
            const int nch = (nb + KC - 1) / KC;
            for (int ch = 0; ch < nch && ok; ++ch, ++g) {
                const int stage = g % NS;
                const int k0 = ch * KC, k1 = min(k0 + KC, nb);
                const int s_lo = oslot[k0], s_hi = oslot[k1 - 1];
                // staging row of chunk column k: rbase + k
                const int rbase = ring ? (k0 & (RING - 1)) : 0;
                // phase 1: orbital values at all points -> staging rows
                if (ring) {
                    // at the first chunk of each group: the slots starting in the group's chunks
                    const int e1 = min(k0 + EG * KC, nb);
                    const int s_first = ps[s_lo].off >= k0 ? s_lo : s_lo + 1;
                    const int nsc = ch % EG == 0 ? oslot[e1 - 1] - s_first + 1 : 0;
                    for (int w = pt; w < kMaxBatchPts * nsc; w += kProd) {
                        const int p = w % kMaxBatchPts, s = s_first + w / kMaxBatchPts;
                        const PSlot sl = ps[s];
                        float *col = stg + p;
                        if (p < npb) {
                            float dx, dy, dz;
                            disp(sl, poff + 6 * p, dx, dy, dz);
                            eval_phi_f32<true>(spec[sl.species], P.coef32, dx, dy, dz, [&](int o, float v) {
                                col[((sl.off + o) & (RING - 1)) * kMaxBatchPts] = v;
                            });
                        } else {
                            for (int o = 0; o < sl.norb; ++o) col[((sl.off + o) & (RING - 1)) * kMaxBatchPts] = 0.f;
                        }
                    }
                } else {
                    const int nsc = s_hi - s_lo + 1;
                    for (int w = pt; w < kMaxBatchPts * nsc; w += kProd) {
                        const int p = w % kMaxBatchPts, s = s_lo + w / kMaxBatchPts;
                        const PSlot sl = ps[s];
                        float *col = stg + p;
                        const int base_k = sl.off - k0;
                        if (p < npb) {
                            float dx, dy, dz;
                            disp(sl, poff + 6 * p, dx, dy, dz);
                            eval_phi_f32<true>(spec[sl.species], P.coef32, dx, dy, dz, [&](int o, float v) {
                                const int k = base_k + o;
                                if (k >= 0 && k < KC) col[k * kMaxBatchPts] = v;
                            });
                        } else {
                            for (int o = 0; o < sl.norb; ++o) {
                                const int k = base_k + o;
                                if (k >= 0 && k < KC) col[k * kMaxBatchPts] = 0.f;
                            }
                        }
                    }
                }
                // columns past the last orbital of the batch (last chunk only)
                for (int w = pt; w < (KC - (k1 - k0)) * kMaxBatchPts; w += kProd)
                    stg[(rbase + k1 - k0) * kMaxBatchPts + w] = 0.f;
                // gather tables of the chunk: element (nu, k) of B is DM32[gbase[b][k] + o_nu * gna[k]]
                // with b the slot of nu (gbase = -1: no block, or k past the last orbital)
                for (int w = pt; w < ns * KC; w += kProd) {
                    const int k = w % KC, b = w / KC;
                    const int mu = k0 + k;
                    int v = -1;
                    if (mu < nb) {
                        const int a = oslot[mu];
                        const int e = tsm ? rtbl[b * ns + a] : __ldg(tbl + b * ns + a);
                        if (e >= 0) v = (e >> 1) + oidx[mu];
                    }
                    gbase[w] = v;
                }
                for (int k = pt; k < KC; k += kProd) gna[k] = (k0 + k < nb) ? ps[oslot[k0 + k]].norb : 0;
                if (g >= NS) ok = role_wait(&empty[stage], ((g / NS) - 1) & 1, P, pt, pflag, 1, kProd);
                else named_sync(1, kProd);
                if (!ok) break;
                unsigned char *base = sm + stage * L::STAGE;
                // phase 2a: A = Phi (rows = points, K = orbitals of the chunk)
                for (int w = pt; w < kMaxBatchPts * S::KCM; w += kProd) {
                    const int p = w % kMaxBatchPts, kc = w / kMaxBatchPts;
                    unsigned char *da[S::NT];
#pragma unroll
                    for (int t = 0; t < S::NT; ++t) da[t] = base + t * L::ARR_A + cm_off<S>(p, kc);
                    float x[S::CG];
#pragma unroll
                    for (int i = 0; i < S::CG; ++i) x[i] = stg[(rbase + kc * S::CG + i) * kMaxBatchPts + p];
                    if constexpr (S::HALF)
#pragma unroll
                        for (int i = 0; i < S::CG; ++i) x[i] *= sA;
                    split_store<S>(x, da);
                }
                // phase 2b: B = D rows nu (N), K = orbitals mu of the chunk: D(b_nu, a_mu)[o_nu][o_mu]
                // read in FP32 through the chunk tables; GB tasks per thread, loads issued first
                // (five 4-wide tasks cover a 220-column chunk in one round without spills)
                constexpr int GB = S::CG == 4 ? 5 : 4;
                for (int w0 = pt; w0 < npad * S::KCM; w0 += kProd * GB) {
                    float x[GB][S::CG];
#pragma unroll
                    for (int gq = 0; gq < GB; ++gq) {
                        const int w = w0 + gq * kProd;
                        const int kc = w % S::KCM, nu = w / S::KCM;
                        const bool rv = w < npad * S::KCM && nu < nb;
                        const int b = rv ? oslot[nu] : 0, ob = rv ? oidx[nu] : 0;
                        const int *gb = gbase + b * KC + kc * S::CG;
                        const int *gn = gna + kc * S::CG;
#pragma unroll
                        for (int i = 0; i < S::CG; ++i) {
                            const int bs = gb[i];
                            x[gq][i] = (rv && bs >= 0) ? __ldg(DM + bs + ob * gn[i]) : 0.f;
                        }
                    }
#pragma unroll
                    for (int gq = 0; gq < GB; ++gq) {
                        const int w = w0 + gq * kProd;
                        if (w >= npad * S::KCM) break;
                        const int kc = w % S::KCM, nu = w / S::KCM;
                        unsigned char *db[S::NT];
#pragma unroll
                        for (int t = 0; t < S::NT; ++t)
                            db[t] = base + S::NT * L::ARR_A + t * L::ARR_B + cm_off<S>(nu, kc);
                        if constexpr (S::HALF)
#pragma unroll
                            for (int i = 0; i < S::CG; ++i) x[gq][i] *= sD;
                        split_store<S>(x[gq], db);
                    }
                }
                fence_async_smem();
                named_sync(1, kProd);
                if (pt == 0) mbar_arrive(&full[stage]);   // chunk g is in shared memory
            }
        }
    } else if (tid < kEpi0) {
        // ------------------------------------------------------------ MMA issue (one thread)
        if (tid == kMma) {
            int g = 0, it = 0;
            bool ok = true;
            CtaRange cr(P);
            for (int bi = 0; ok && cr.next(bi);) {
                const int nb = P.batches[bi].nb;
                if (nb == 0) continue;
                const int npad = (nb + 15) & ~15;
                const int buf = it & 1;
                const int nch = (nb + KC - 1) / KC;
                const uint32_t id = idesc<S>(128, npad);
                for (int ch = 0; ch < nch && ok; ++ch, ++g) {
                    const int stage = g % NS;
                    ok = !aborted(P) && mbar_wait(&full[stage], (g / NS) & 1, P.spin_limit);
                    if (ok && ch == 0 && it >= 2)   // the epilogue of batch it - 2 is done
                        ok = !aborted(P) && mbar_wait(&accempty[buf], ((it >> 1) - 1) & 1, P.spin_limit);
                    if (!ok) {
                        report_timeout(P);
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a0 = su32(sm + stage * L::STAGE), b0 = a0 + S::NT * L::ARR_A;
#pragma unroll
                    for (int ks = 0; ks < S::KCM / 2; ++ks) {
#pragma unroll
                        for (int q = 0; q < S::NPROD; ++q) {
                            const uint64_t da = sdesc(a0 + term(S::PA, q) * L::ARR_A + ks * 2 * kLBO, SBO);
                            const uint64_t db = sdesc(b0 + term(S::PB, q) * L::ARR_B + ks * 2 * kLBO, SBO);
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
        // warp (q, hh): TMEM lane quadrant q (points 32q..32q+31), atom images s with s % 2 == hh
        const int et = tid - kEpi0, ew = et >> 5, lane = et & 31;
        const int q = ew & 3, hh = ew >> 2;
        const int p = q * 32 + lane;  // TMEM lane = point of the batch
        float *w = win + ew * kWin * 32;
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
            named_sync(2, kEpi);
            load_geom(P, SI, B, eps, epoff, et, kEpi);
            if (FORCE)
                for (int e = et; e < 3 * ns; e += kEpi) facc[e] = 0.f;
            if (!role_wait(&accfull[buf], (it >> 1) & 1, P, et, eflag, 2, kEpi)) break;
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
            int w0 = -1000, wn = 0;
            for (int s = hh; s < ns; s += 2) {
                const PSlot sl = eps[s];
                float fx = 0.f, fy = 0.f, fz = 0.f;
                float dx = 0.f, dy = 0.f, dz = 0.f;
                if (pv) disp(sl, po, dx, dy, dz);
                // a point outside the image's sphere adds nothing: skip its evaluation (the
                // window loads below stay warp-uniform)
                const bool in = pv && dx * dx + dy * dy + dz * dz < spec[sl.species].rcut2;
                // orbitals [oa, ob) of the slot whose columns fit the window (all of them unless
                // the slot has more than 17 orbitals)
                for (int oa = 0; oa < sl.norb;) {
                    const int ob = min(sl.norb, ((sl.off + oa) & ~15) + kWin - sl.off);
                    if (sl.off + oa < w0 || sl.off + ob > w0 + wn) {
                        w0 = (sl.off + oa) & ~15;
                        wn = ((sl.off + ob - w0) + 15) & ~15;
                        for (int c = 0; c < wn; c += 16) {
                            float v[16];
                            tmem_ld16(trow + (uint32_t)(w0 + c), v);
#pragma unroll
                            for (int j = 0; j < 16; ++j) w[(c + j) * 32 + lane] = v[j];
                        }
                    }
                    const int cb = sl.off - w0;   // window column of orbital o: cb + o
                    if (in) {
                        if (FORCE)
                            eval_phigrad_f32(spec[sl.species], P.coef32, dx, dy, dz,
                                             [&](int o, float v, float gx, float gy, float gz) {
                                                 if (o >= oa && o < ob) {
                                                     const float y = w[(cb + o) * 32 + lane];
                                                     racc += v * y;
                                                     fx += gx * y; fy += gy * y; fz += gz * y;
                                                 }
                                             });
                        else
                            eval_phi_f32(spec[sl.species], P.coef32, dx, dy, dz, [&](int o, float v) {
                                if (o >= oa && o < ob) racc += v * w[(cb + o) * 32 + lane];
                            });
                    }
                    oa = ob;
                }
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
                        // the four lane quadrants of a slot meet here: FP32 shared-memory adds
                        // (native), FP64 from the per-batch sum on
                        atomicAdd(&facc[3 * s + 0], fx);
                        atomicAdd(&facc[3 * s + 1], fy);
                        atomicAdd(&facc[3 * s + 2], fz);
                    }
                }
            }
            tc_fence_before();
            mbar_arrive(&accempty[buf]);
            racc *= u;
            if (RHO && hh == 1) rpart[p] = racc;
            named_sync(2, kEpi);
            if (RHO && hh == 0 && pv) SI.rho[gi] = f2d(racc + rpart[p]);
            if (FORCE && SI.F)
                for (int e = et; e < 3 * ns; e += kEpi)
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
    k_vlocal_tc<S><<<grid, kThreadsTC, smem, s>>>(P, si0, sis, max_nb <= 192 ? 2 : 1);
    return cudaGetLastError();
}

template <class S, bool R, bool Fo, bool St>
cudaError_t rho_launch3(const Plan &P, const SInfo &si0, const SInfo *sis, cudaStream_t s, int nsm)
{
    constexpr int smem = RSmem<S>::TOTAL;
    static_assert(smem <= 232448, "rho shared memory");
    cudaError_t e = set_smem(k_rho_tc<S, R, Fo, St>, smem);
    if (e != cudaSuccess) return e;
    const int grid = P.rng ? P.npart : std::min(nsm, P.nbatches);
    k_rho_tc<S, R, Fo, St><<<grid, kThreadsTC, smem, s>>>(P, si0, sis);
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
