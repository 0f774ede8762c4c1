// Internal data structures shared by the host set-up and the CUDA kernels of libgint.
#pragma once
#include <cstdint>
#include <memory>
#include <string>
#include <utility>
#include <vector>

#include <cuda_runtime.h>

#include "../../include/gint.h"

namespace gint {

constexpr int kMaxRad = 16;        // radial functions per species
constexpr int kMaxSpecies = 8;
constexpr int kMaxOrbSpecies = 48; // orbitals per species (l <= 2)
constexpr int kMaxNb = 256;        // orbitals per batch (tensor-memory columns of one tile pair)
constexpr int kMaxSlots = 64;      // atom images per batch
constexpr int kMaxBatchPts = 128;  // grid points per batch
constexpr int kMaxBatchDim = 16;   // points per batch along one axis

// One species as the kernels see it.  Orbital o of the species belongs to radial rad_of[o]
// with harmonic index m_of[o] in 0..2l (order m = 0, +1, -1, +2, -2).
struct DevSpecies {
    int nrad, norb, nint;          // nint = ntab - 1 spline intervals
    int coef_off;                  // first interval record of this species (see Plan::coef*)
    int env_off;                   // first entry of this species in Plan::env
    double rcut, inv_dr;
    float rcut_f, inv_dr_f;
    int l[kMaxRad];
};

// A grid batch: points (i0 + a, j0 + b, k0 + c) for a < n1, b < n2, c < n3 (k fastest inside
// the batch), its atom images slot0 .. slot0+nslots-1 and orbital count nb.
struct Batch {
    int i0, j0, k0;
    int dims;                      // n1 | n2 << 8 | n3 << 16 | structure id << 24
    int slot0, nslots, nb;
    int tbl;                       // first entry of this batch's nslots x nslots pair tables
                                   //   (BatchSet::tbl in tbl_index order, tbl2 row-major)
};

// An atom image seen by a batch.  d0 = (grid point (i0,j0,k0)) - (tau_I + R_a), Cartesian,
// in FP64 and as an FP32 pair (dh + dl) for the FP32 kernels.
struct Slot {
    int atom, species, orb_off, norb;
    double d0[3];
    float dh[3], dl[3];
};

// The fields of a Slot that the tensor-core kernels read, as a 40-byte record of its own array
// (a batch's records then span 5/8 of the memory sectors of its Slot records).
struct TSlot {
    int atom, species, orb_off, norb;
    float dh[3], dl[3];
};

constexpr int kPoffDim = 16;       // point-offset table covers local indices 0..15 per axis
constexpr long long kDrainBudget = 4000000000LL;  // final wait for in-flight MMAs (clock cycles)

// Per-structure data of the tensor-core kernels: the buffers of one call and the grid.  A
// single-structure launch passes one by value; a batched launch reads them from device memory
// by the structure id of each batch.
struct SInfo {
    const double *V;
    double *H;
    const void *DMS;               // split density matrix (k_dm_split): every block's NT terms,
                                   //   rows and columns padded, at element NT x its split offset
    int64_t dms_plane;
    int padn;                      // the split store's layout (padded, or row layout) and N columns
    double *rho;
    double *F;
    double *dLde;                  // 9 values: strain derivative (single-structure launches only)
    const float *poff;
    int grid[3];
    float phimax;                  // bound on |phi| over the species (fp16 operand scaling)
    double dV;
    const float *amax;             // device [2]: max |V(r)| and max |density matrix| of the call,
                                   // written before the kernel by the fp16 path (else unused)
    float hstep[9];                // grid step vectors a_i / N_i of this structure (FP32)
};

// Everything a kernel needs, passed by value.
struct Plan {
    int natoms, nspecies;
    int grid[3];
    int64_t npts;
    int nbatches;
    double dV;
    double h[9];                   // h[3*i + c] = component c of a_i / N_i
    DevSpecies sp[kMaxSpecies];
    const double *coef64;          // [interval record][4]: per species, interval-major, radial-minor
    const float4 *coef32;
    const float *env;              // per species and interval i: a bound on |phi| at r >= i dr
    const Batch *batches;
    const Slot *slots;
    const TSlot *tslots;           // the same atom images, the tensor-core kernels' fields
    const int *tbl;                // (block offset << 1 | canonical) or -1 if no block
    const int *koff;               // per slot: padded K column (density kernel)
    const int *tbl2;               // per slot pair: split density-matrix block offset or -1
    const float *poff;             // [16][16][16][6]: a h1 + b h2 + c h3 as FP32 hi (3) + lo (3)
    const int *partner;            // [nblocks] partner block index
    const int64_t *blk_off;        // [nblocks + 1]
    const int *blk_rows;           // [nblocks] rows of each block
    int64_t nblocks, nvalues;
    int *status;                   // device status word
    long long spin_limit;          // clock64 cycles a kernel may wait on one pipeline barrier
    const int2 *rng;               // [nseg][npart]: batch range [x, y) of each CTA of a persistent
    int npart, nseg;               //   launch per segment, or null for equal counts per CTA
};

// One decomposition of the grid into batches, with its atom-image lists and pair tables.
// Padded K layout of a batch's orbitals for the tensor-core density kernel: every slot's orbital
// count is rounded up to kKPad columns, and a slot that fits kKSeg columns never crosses a
// multiple of kKSeg (it starts at the next one instead), so the operand pieces of 16 bytes and
// the staging segments of one producer task each belong to one slot.
constexpr int kKPad = 8;
constexpr int kKSeg = 16;
constexpr int kMaxKCols = 4096;        // padded K columns of one batch
__host__ __device__ constexpr int kpad(int norb) { return (norb + kKPad - 1) / kKPad * kKPad; }

// Allocator whose resize leaves new elements of trivial types uninitialised: the set-up writes
// every element of its large per-batch arrays itself, so a zero fill would only cost time.
template <class T>
struct DefaultInit : std::allocator<T> {
    template <class U>
    struct rebind {
        using other = DefaultInit<U>;
    };
    DefaultInit() = default;
    template <class U>
    DefaultInit(const DefaultInit<U> &) {}
    template <class U, class... A>
    void construct(U *p, A &&...a)
    {
        if constexpr (sizeof...(A) == 0)
            ::new ((void *)p) U;
        else
            ::new ((void *)p) U(std::forward<A>(a)...);
    }
};
template <class T>
using hvec = std::vector<T, DefaultInit<T>>;

// Block key -> block index: open addressing over the packed keys (I, J, n), which are >= 0.
struct KeyIndex {
    std::vector<int64_t> key;
    std::vector<int> val;
    uint64_t mask = 0;
    KeyIndex() = default;
    explicit KeyIndex(const std::vector<int64_t> &packed)
    {
        size_t cap = 16;
        while (cap < 2 * packed.size()) cap <<= 1;
        key.assign(cap, -1);
        val.assign(cap, -1);
        mask = cap - 1;
        for (size_t i = 0; i < packed.size(); ++i) {
            uint64_t h = slot_of(packed[i]);
            while (key[h] != -1) h = (h + 1) & mask;
            key[h] = packed[i];
            val[h] = (int)i;
        }
    }
    uint64_t slot_of(int64_t k) const { return ((uint64_t)k * 0x9E3779B97F4A7C15ull >> 17) & mask; }
    int find(int64_t k) const
    {
        for (uint64_t h = slot_of(k);; h = (h + 1) & mask) {
            if (key[h] == k) return val[h];
            if (key[h] == -1) return -1;
        }
    }
};

// Entry of slot pair (a, b) in a batch's ns x ns slot-pair table (Batch::tbl): the upper
// triangle a <= b first, row by row, then the strictly lower triangle row by row, so that the
// tensor-core scatter, which reads only pairs a <= b, reads one contiguous range.
__host__ __device__ inline int tbl_index(int a, int b, int ns)
{
    return a <= b ? a * ns - a * (a - 1) / 2 + (b - a) : ns * (ns + 1) / 2 + a * (a - 1) / 2 + b;
}

struct BatchSet {
    int dims[3] = {0, 0, 0};
    hvec<Batch> batches;
    hvec<Slot> slots;
    hvec<int> slot_img;              // 3 per slot: image n of the slot's atom
    hvec<int> tbl;                   // per slot pair (a, b), at tbl_index(a, b, ns): block
                                     //   offset << 1 | canonical, or -1
    hvec<int> koff;                  // per slot: first column in the padded K layout
    hvec<int> tbl2;                  // per slot pair (b, a): offset of block (b, a) in the split
                                     //   density-matrix store, or -1 (rho/force set only)
    int limit_nb = 256;              // batches with more orbitals are split
    bool padn = false;               // rho/force: N columns at the padded K offsets, padded
                                     //   density layout (otherwise N = the unpadded orbitals)
    bool shared = false;             // rho/force: the lists, tables and offsets are copies of the
                                     //   vlocal ones (same batch shape; only tbl2 is its own)
    int max_nb = 0, max_slots = 0;
    int max_k = 0;                   // largest padded K of a batch
    double flops_dense = 0.0;
    std::vector<int2> rng;           // cost-balanced CTA ranges of the persistent kernels
    void *d_batches = nullptr, *d_slots = nullptr, *d_tbl = nullptr, *d_rng = nullptr;
    void *d_koff = nullptr, *d_tbl2 = nullptr;
    void *d_tslots = nullptr;
    size_t d_cap[7] = {0, 0, 0, 0, 0, 0, 0};   // bytes allocated for d_batches, d_slots, d_tbl, d_rng,
                                             //   d_koff, d_tbl2, d_tslots
};

// Split batches [0, n) into at most nparts contiguous ranges of about equal estimated cost
// (kind 0: vlocal, 1: rho/force); returns the nparts' + 1 range bounds.
std::vector<int> partition_batches(const Batch *b, size_t n, int nparts, int kind);

// CTA ranges of a persistent launch of npart CTAs over consecutive segments [seg[i], seg[i+1])
// of a batch list: each segment is split by cost over min(npart, its batches) CTAs, the CTAs
// that receive work rotating from one segment to the next; other CTAs get an empty range.
std::vector<int2> segment_ranges(const Batch *b, const std::vector<int> &seg, int npart, int kind);

}  // namespace gint

struct gint_handle_s {
    gint::Plan plan{};
    int device = 0;
    int nsm = 0;
    // host copies
    double cell[9];
    int grid[3];
    int natoms = 0, nspecies = 0;
    std::vector<int> species;
    std::vector<double> tau;
    std::vector<int> norb_atom;
    std::vector<int32_t> keys;       // 5 per block
    std::vector<int64_t> offsets;    // nblocks + 1
    std::vector<int> partner;
    std::vector<uint8_t> canon;      // per block: the canonical member of its partner pair
    gint::KeyIndex kidx;             // block key -> block index
    gint::BatchSet bs[2];            // [0] vlocal batches, [1] rho/force batches
    gint::BatchSet spare[2];         // host arrays of the lists a position update replaced, kept
                                     //   (allocated and touched) for the next update to write into
    gint::hvec<gint::TSlot> tslot_stage;  // host staging of the tensor-core slot records (upload)
    bool relist[2] = {false, false}; // a position update changed that decomposition's lists
    bool flops_stale = false;        // info.flops_useful predates the last position update
    std::vector<float4> coef32_host; // spline records, as uploaded
    std::vector<float> env_host;     // |phi| envelopes, as uploaded
    void *d_env = nullptr;
    gint_options opt{};
    gint_info_t info{};
    // device memory (owned)
    void *d_coef64 = nullptr, *d_coef32 = nullptr;
    void *d_partner = nullptr, *d_blkoff = nullptr, *d_blkrows = nullptr;
    int *d_status = nullptr;
    double *d_dmsym = nullptr;       // scratch: block-symmetrised density matrix (FP64 kernels)
    void *d_dms = nullptr;           // scratch: split density matrix of the tensor-core kernels
    int64_t dms_plane = 0;           // elements per term of it (Sum_b kpad(n_I) kpad(n_J) in the padded
                                     //   layout, Sum_b n_I kpad(n_J) in the row layout; rounded to 8)
    std::vector<int> soff;           // per block: offset in a plane of the split store
    void *d_soff = nullptr;
    float *d_poff = nullptr;         // point-offset table
    double *d_red = nullptr;         // scratch: partial sums of reductions
    float *d_amax = nullptr;         // scratch: largest |V(r)| and |DM| of an fp16 call (2 floats)
    float phimax = 1.f;              // bound on |phi_mu(r)| from the spline records
    struct {                         // k-space transforms (built on first use)
        int *d_keys = nullptr;       // [nblocks][5] block keys
        int *d_grp = nullptr;        // [ngroups + 1] first block of each (I, J) group
        int *d_pair = nullptr;       // [natoms * natoms] group of atom pair (I, J), -1 if none
        int *d_colatom = nullptr;    // [nbasis] atom of each orbital (dense column)
        int *d_orboff = nullptr;     // [natoms + 1] orbital offsets (atom-major)
        int ngroups = 0;
        double *d_kvec = nullptr;    // [cap][4]: kappa (3) and weight of each k point
        double *d_phase = nullptr;   // [nblocks][cap][2]: cos, sin of 2 pi kappa.n
        int cap = 0;
    } ks;
    double *d_dm_scratch = nullptr;  // dense rho(k), planar real / imaginary (gint_density_matrix)
    size_t dm_scratch_bytes = 0;
    float *d_dm_planes = nullptr;    // TF32 hi / lo operand planes of the tensor-core density matrix
    size_t dm_planes_bytes = 0;
    double *d_hostio = nullptr;      // buffers of gint_run_host (allocated on first use)
    size_t hostio_bytes = 0;
    cudaStream_t io_stream = nullptr; // gint_run_host's copy stream and its events (first use)
    cudaEvent_t io_ev[4] = {nullptr, nullptr, nullptr, nullptr};
    cudaStream_t last_stream = nullptr;
};

namespace gint {
// kernel parameters for one batch decomposition (0 = vlocal, 1 = rho/force)
inline Plan plan_for(const gint_handle_s *h, int which)
{
    Plan p = h->plan;
    const BatchSet &b = h->bs[which];
    p.batches = (const Batch *)b.d_batches;
    p.slots = (const Slot *)b.d_slots;
    p.tslots = (const TSlot *)b.d_tslots;
    p.tbl = (const int *)b.d_tbl;
    p.koff = (const int *)b.d_koff;
    p.tbl2 = (const int *)b.d_tbl2;
    p.nbatches = (int)b.batches.size();
    p.rng = (const int2 *)b.d_rng;
    p.npart = (int)b.rng.size();
    p.nseg = 1;
    return p;
}
void set_error(const char *fmt, ...);
gint_status cuda_fail(cudaError_t e, const char *where);
// GINT_EINVAL (with the message set) unless h is non-null and its device is the current one
gint_status check_handle(gint_handle h, const char *who);
// set-up helpers (gint_setup.cpp)
// old: the handle whose positions are being updated (its block list must stay the same), or
// nullptr at set-up
gint_status build_geometry(gint_handle h, const double *tau, const gint_handle_s *old);
// kernel launchers (gint_simt.cu, gint_tc.cu, gint_api.cu)
cudaError_t launch_vlocal_simt(const Plan &p, bool fp64, const double *V, double *H, cudaStream_t s, int nsm);
cudaError_t launch_rho_force_simt(const Plan &p, bool fp64, const double *V, const double *DM,
                                  double *rho, double *F, double *dLde, cudaStream_t s, int nsm);
cudaError_t launch_vlocal_tc(const Plan &p, gint_prec prec, const SInfo &si0, const SInfo *sis, cudaStream_t s,
                             int nsm, int max_nb);
// NT terms of the (block-symmetrised if sym) density matrix into the padded split store
// the handle's split density-matrix store (padded or row layout, see k_dm_split)
cudaError_t launch_dm_split(const Plan &P, gint_prec prec, const int *soff, const double *DM, void *out,
                            int64_t plane, bool padn, bool sym, const float *amax, cudaStream_t s);
cudaError_t launch_absmax(const double *x, int64_t n, float *out, cudaStream_t s);
cudaError_t launch_rho_force_tc(const Plan &p, gint_prec prec, const SInfo &si0, const SInfo *sis, bool rho,
                                bool force, cudaStream_t s, int nsm);
// the single-structure SInfo of a handle for one call
SInfo sinfo_for(const gint_handle_s *h, const double *V, double *H, const void *DMS, double *rho, double *F);
}  // namespace gint
