// Multi-structure jobs (gint_batch_*), the one-shot gint_batched, and the batch-shape
// autotuner (gint_autotune).
//
// Many structures of uneven size are independent grid integrations (the grid partition of
// Sec. IV.B extended across structures).  A job concatenates the batch decompositions of all
// structures into one work list; each batch record carries its structure id, through which
// the tensor-core kernels find that structure's buffers, grid and point offsets.  One
// persistent launch of each kernel then covers every structure, and the whole sequence is
// captured once into a CUDA graph.
#include <algorithm>
#include <cstring>
#include <vector>

#include "gint_internal.h"

using namespace gint;

namespace gint {
cudaError_t launch_mirror(const Plan &P, double *H, cudaStream_t s);
}

static bool tc_prec(gint_prec p)
{
    return p == GINT_TF32X3 || p == GINT_BF16X3 || p == GINT_BF16X6 || p == GINT_FP16X3;
}

struct gint_batch_s {
    int nstruct = 0;
    gint_prec prec = GINT_TF32X3;
    int device = 0;
    int nsm = 0;
    bool with_rho = false;
    std::vector<gint_handle> hs;
    std::vector<const double *> V, DM;
    std::vector<double *> H, rho;
    Plan plan[3];                    // combined plans: [0] vlocal (batches <= 192 orbitals),
                                     // [1] rho, [2] vlocal of structures with larger batches
    int max_nb_v[3] = {0, 0, 0};
    void *d_mem[25] = {nullptr};    // [3w..3w+2] batches, slots, tables; [9] splines; [12+w] CTA ranges;
                                     // [15+2w], [16+2w] padded K offsets and split-store tables;
                                     // [21] |phi| envelopes; [22+w] tensor-core slot records
    SInfo *d_sinfo = nullptr;
    int *d_status = nullptr;
    float *d_amax = nullptr;         // [2 * nstruct]: max |V| and max |DM| of each entry (fp16 path)
    std::vector<void *> dms;         // split density matrix of each entry: the handle's scratch for
    std::vector<void *> own;         //   its first occurrence, a private buffer for repeats
    cudaStream_t cap = nullptr;
    cudaGraph_t graph = nullptr;
    cudaGraphExec_t exec = nullptr;
};

namespace {

template <class T>
cudaError_t upload_vec(void **dst, const std::vector<T> &v)
{
    cudaError_t e = cudaMalloc(dst, std::max<size_t>(sizeof(T), v.size() * sizeof(T)));
    if (e != cudaSuccess) return e;
    return v.empty() ? cudaSuccess : cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
}

void free_batch(gint_batch b)
{
    if (b->exec) cudaGraphExecDestroy(b->exec);
    if (b->graph) cudaGraphDestroy(b->graph);
    if (b->cap) cudaStreamDestroy(b->cap);
    for (void *p : b->d_mem)
        if (p) cudaFree(p);
    for (void *p : b->own)
        if (p) cudaFree(p);
    if (b->d_sinfo) cudaFree(b->d_sinfo);
    if (b->d_status) cudaFree(b->d_status);
    if (b->d_amax) cudaFree(b->d_amax);
    delete b;
}

bool same_species(const gint_handle a, int sa, const gint_handle b, int sb)
{
    const DevSpecies &x = a->plan.sp[sa], &y = b->plan.sp[sb];
    if (x.nrad != y.nrad || x.nint != y.nint || x.rcut != y.rcut || x.inv_dr != y.inv_dr) return false;
    for (int r = 0; r < x.nrad; ++r)
        if (x.l[r] != y.l[r]) return false;
    const size_t n = (size_t)x.nint * x.nrad;
    return std::memcmp(&a->coef32_host[x.coef_off], &b->coef32_host[y.coef_off], n * sizeof(float4)) == 0;
}

// the job's launch sequence on stream s (captured into the graph)
gint_status issue(gint_batch b, cudaStream_t s)
{
    cudaError_t e;
    const bool half = b->prec == GINT_FP16X3;
    if (half && (e = cudaMemsetAsync(b->d_amax, 0, sizeof(float) * 2 * b->nstruct, s)) != cudaSuccess)
        return cuda_fail(e, "gint_batch: memset");
    for (int i = 0; i < b->nstruct; ++i) {
        gint_handle h = b->hs[i];
        if ((e = cudaMemsetAsync(b->H[i], 0, sizeof(double) * h->info.nvalues, s)) != cudaSuccess)
            return cuda_fail(e, "gint_batch: memset");
        if (half && (e = launch_absmax(b->V[i], h->info.npts, b->d_amax + 2 * i, s)) != cudaSuccess)
            return cuda_fail(e, "gint_batch: potential range");
        if (b->with_rho && h->info.nvalues > 0) {
            float *am = half ? b->d_amax + 2 * i + 1 : nullptr;
            if (am && (e = launch_absmax(b->DM[i], h->info.nvalues, am, s)) != cudaSuccess)
                return cuda_fail(e, "gint_batch: density-matrix range");
            if ((e = launch_dm_split(h->plan, b->prec, (const int *)h->d_soff, b->DM[i], b->dms[i], h->dms_plane,
                                     h->bs[1].padn, false, am, s)) != cudaSuccess)
                return cuda_fail(e, "gint_batch: split");
        }
    }
    SInfo none{};
    // structures whose vlocal batches fit two TMEM accumulators run in one persistent launch,
    // the others (some batch over 192 orbitals) in a second one with a single accumulator
    for (int w : {0, 2})
        if (b->plan[w].nbatches > 0 &&
            (e = launch_vlocal_tc(b->plan[w], b->prec, none, b->d_sinfo, s, b->nsm, b->max_nb_v[w])) != cudaSuccess)
            return cuda_fail(e, "gint_batch: vlocal");
    for (int i = 0; i < b->nstruct; ++i)
        if ((e = launch_mirror(b->hs[i]->plan, b->H[i], s)) != cudaSuccess) return cuda_fail(e, "gint_batch: mirror");
    if (b->with_rho &&
        (e = launch_rho_force_tc(b->plan[1], b->prec, none, b->d_sinfo, true, false, s, b->nsm)) != cudaSuccess)
        return cuda_fail(e, "gint_batch: rho");
    return GINT_OK;
}

}  // namespace

extern "C" gint_status gint_batch_create(gint_batch *out, int nstruct, const gint_handle *hs, const double *const *V,
                                         double *const *H, const double *const *DM, double *const *rho,
                                         gint_prec prec)
{
    if (!out || nstruct < 1 || nstruct > 255 || !hs || !V || !H || !tc_prec(prec)) {
        set_error("gint_batch_create: need 1..255 structures, V and H arrays, and a tensor-core precision");
        return GINT_EINVAL;
    }
    *out = nullptr;
    int dev = -1;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "gint_batch_create");
    const bool with_rho = DM && rho;
    for (int i = 0; i < nstruct; ++i) {
        if (!hs[i] || hs[i]->device != dev || !V[i] || !H[i] || (with_rho && (!DM[i] || !rho[i]))) {
            set_error("gint_batch_create: structure %d: null handle/buffer or handle on another device", i);
            return GINT_EINVAL;
        }
    }
    gint_batch b = new gint_batch_s();
    b->nstruct = nstruct;
    b->prec = prec;
    b->device = dev;
    b->nsm = hs[0]->nsm;
    b->with_rho = with_rho;
    b->hs.assign(hs, hs + nstruct);
    b->V.assign(V, V + nstruct);
    b->H.assign(H, H + nstruct);
    if (with_rho) {
        b->DM.assign(DM, DM + nstruct);
        b->rho.assign(rho, rho + nstruct);
    }
    // merged species and spline records
    Plan base = hs[0]->plan;
    std::vector<float4> coef;
    std::vector<float> env;
    std::vector<std::pair<int, int>> uniq;  // (handle, species) of each merged species
    std::vector<std::vector<int>> remap(nstruct);
    int nsp = 0;
    for (int i = 0; i < nstruct; ++i) {
        remap[i].resize(hs[i]->nspecies);
        for (int s = 0; s < hs[i]->nspecies; ++s) {
            int found = -1;
            for (int u = 0; u < nsp && found < 0; ++u)
                if (same_species(hs[uniq[u].first], uniq[u].second, hs[i], s)) found = u;
            if (found < 0) {
                if (nsp == kMaxSpecies) {
                    free_batch(b);
                    set_error("gint_batch_create: more than %d distinct species", kMaxSpecies);
                    return GINT_EINVAL;
                }
                DevSpecies d = hs[i]->plan.sp[s];
                const size_t n = (size_t)d.nint * d.nrad;
                const int off = (int)coef.size();
                coef.insert(coef.end(), hs[i]->coef32_host.begin() + d.coef_off,
                            hs[i]->coef32_host.begin() + d.coef_off + n);
                d.coef_off = off;
                const int eoff = (int)env.size();
                env.insert(env.end(), hs[i]->env_host.begin() + d.env_off, hs[i]->env_host.begin() + d.env_off + d.nint);
                d.env_off = eoff;
                base.sp[nsp] = d;
                uniq.push_back({i, s});
                found = nsp++;
            }
            remap[i][s] = found;
        }
    }
    base.nspecies = nsp;
    // concatenated batch lists with the structure id in each batch record
    for (int w = 0; w < 3; ++w) {
        std::vector<Batch> bat;
        std::vector<Slot> sl;
        std::vector<TSlot> tsl;
        std::vector<int> tbl, koff, tbl2;
        std::vector<int> seg{0};
        const int src = w == 1 ? 1 : 0;
        for (int i = 0; i < nstruct; ++i) {
            const BatchSet &bs = hs[i]->bs[src];
            if (w == 0 && bs.max_nb > 192) continue;
            if (w == 2 && bs.max_nb <= 192) continue;
            const int s0 = (int)sl.size(), t0 = (int)tbl.size();
            for (Batch B : bs.batches) {
                B.slot0 += s0;
                B.tbl += t0;
                B.dims |= i << 24;
                bat.push_back(B);
            }
            for (Slot S : bs.slots) {
                S.species = remap[i][S.species];
                sl.push_back(S);
                TSlot T;
                T.atom = S.atom;
                T.species = S.species;
                T.orb_off = S.orb_off;
                T.norb = S.norb;
                for (int c = 0; c < 3; ++c) {
                    T.dh[c] = S.dh[c];
                    T.dl[c] = S.dl[c];
                }
                tsl.push_back(T);
            }
            tbl.insert(tbl.end(), bs.tbl.begin(), bs.tbl.end());
            koff.insert(koff.end(), bs.koff.begin(), bs.koff.end());
            tbl2.insert(tbl2.end(), bs.tbl2.begin(), bs.tbl2.end());   // offsets into each entry's own store
            seg.push_back((int)bat.size());
            b->max_nb_v[w] = std::max(b->max_nb_v[w], bs.max_nb);
        }
        if ((e = upload_vec(&b->d_mem[3 * w + 0], bat)) != cudaSuccess ||
            (e = upload_vec(&b->d_mem[3 * w + 1], sl)) != cudaSuccess ||
            (e = upload_vec(&b->d_mem[22 + w], tsl)) != cudaSuccess ||
            (e = upload_vec(&b->d_mem[3 * w + 2], tbl)) != cudaSuccess ||
            (e = upload_vec(&b->d_mem[15 + 2 * w], koff)) != cudaSuccess ||
            (e = upload_vec(&b->d_mem[16 + 2 * w], tbl2)) != cudaSuccess) {
            free_batch(b);
            return cuda_fail(e, "gint_batch_create: upload");
        }
        // one segment per structure: every CTA works on the same structure at about the same
        // time, so the block stores being accumulated stay few (and in L2)
        const std::vector<int2> rng = segment_ranges(bat.data(), seg, b->nsm, w == 1 ? 1 : 0);
        if ((e = upload_vec(&b->d_mem[12 + w], rng)) != cudaSuccess) {
            free_batch(b);
            return cuda_fail(e, "gint_batch_create: upload");
        }
        Plan p = base;
        p.rng = (const int2 *)b->d_mem[12 + w];
        p.npart = b->nsm;
        p.nseg = (int)seg.size() - 1;
        p.batches = (const Batch *)b->d_mem[3 * w + 0];
        p.slots = (const Slot *)b->d_mem[3 * w + 1];
        p.tslots = (const TSlot *)b->d_mem[22 + w];
        p.tbl = (const int *)b->d_mem[3 * w + 2];
        p.koff = (const int *)b->d_mem[15 + 2 * w];
        p.tbl2 = (const int *)b->d_mem[16 + 2 * w];
        p.nbatches = (int)bat.size();
        b->plan[w] = p;
    }
    // a handle may appear more than once (spin channels or several potentials on one geometry):
    // every occurrence after the first gets its own split density-matrix buffer
    b->dms.assign(nstruct, nullptr);
    for (int i = 0; i < nstruct && with_rho; ++i) {
        bool repeat = false;
        for (int j = 0; j < i && !repeat; ++j) repeat = hs[j] == hs[i];
        if (!repeat) {
            b->dms[i] = hs[i]->d_dms;
            continue;
        }
        void *p = nullptr;
        if ((e = cudaMalloc(&p, std::max<size_t>(16, (size_t)hs[i]->dms_plane * 8))) != cudaSuccess) {
            free_batch(b);
            return cuda_fail(e, "gint_batch_create: allocate");
        }
        b->own.push_back(p);
        b->dms[i] = p;
    }
    if ((e = cudaMalloc((void **)&b->d_amax, sizeof(float) * 2 * nstruct)) != cudaSuccess ||
        (e = cudaMemset(b->d_amax, 0, sizeof(float) * 2 * nstruct)) != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "gint_batch_create: allocate");
    }
    std::vector<SInfo> si(nstruct);
    for (int i = 0; i < nstruct; ++i) {
        si[i] = sinfo_for(hs[i], V[i], H[i], with_rho ? b->dms[i] : nullptr, with_rho ? rho[i] : nullptr, nullptr);
        si[i].amax = b->d_amax + 2 * i;
    }
    if ((e = upload_vec(&b->d_mem[9], coef)) != cudaSuccess || (e = upload_vec(&b->d_mem[21], env)) != cudaSuccess ||
        (e = upload_vec((void **)&b->d_sinfo, si)) != cudaSuccess ||
        (e = cudaMalloc((void **)&b->d_status, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(b->d_status, 0, sizeof(int))) != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "gint_batch_create: upload");
    }
    for (int w = 0; w < 3; ++w) {
        b->plan[w].coef32 = (const float4 *)b->d_mem[9];
        b->plan[w].env = (const float *)b->d_mem[21];
        b->plan[w].status = b->d_status;
    }
    // capture the launch sequence once
    if ((e = cudaStreamCreateWithFlags(&b->cap, cudaStreamNonBlocking)) != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "gint_batch_create: stream");
    }
    if ((e = cudaStreamBeginCapture(b->cap, cudaStreamCaptureModeRelaxed)) != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "gint_batch_create: begin capture");
    }
    gint_status st = issue(b, b->cap);
    e = cudaStreamEndCapture(b->cap, &b->graph);
    if (st != GINT_OK) {
        free_batch(b);
        return st;
    }
    if (e != cudaSuccess || (e = cudaGraphInstantiate(&b->exec, b->graph, 0)) != cudaSuccess) {
        free_batch(b);
        return cuda_fail(e, "gint_batch_create: graph");
    }
    *out = b;
    return GINT_OK;
}

extern "C" gint_status gint_batch_launch(gint_batch b, void *stream)
{
    if (!b) {
        set_error("gint_batch_launch: null job");
        return GINT_EINVAL;
    }
    cudaError_t e = cudaGraphLaunch(b->exec, (cudaStream_t)stream);
    if (e != cudaSuccess) return cuda_fail(e, "gint_batch_launch");
    for (gint_handle h : b->hs) h->last_stream = (cudaStream_t)stream;
    return GINT_OK;
}

extern "C" gint_status gint_batch_destroy(gint_batch b)
{
    if (b) free_batch(b);
    return GINT_OK;
}

extern "C" gint_status gint_batched(int nstruct, const gint_handle *hs, const double *const *V, double *const *H,
                                   const double *const *DM, double *const *rho, gint_prec prec, void *stream)
{
    if (nstruct < 0 || (nstruct > 0 && (!hs || !V || !H)) || prec < GINT_FP64 || prec > GINT_FP16X3) {
        set_error("gint_batched: invalid arguments");
        return GINT_EINVAL;
    }
    if (nstruct == 0) return GINT_OK;
    cudaStream_t s = (cudaStream_t)stream;
    if (prec == GINT_FP64 || prec == GINT_FP32) {
        for (int i = 0; i < nstruct; ++i) {
            gint_status st = gint_vlocal(hs[i], V[i], H[i], prec, stream);
            if (st != GINT_OK) return st;
            if (DM && rho && (st = gint_rho(hs[i], DM[i], rho[i], prec, stream)) != GINT_OK) return st;
        }
        return GINT_OK;
    }
    gint_batch b = nullptr;
    gint_status st = gint_batch_create(&b, nstruct, hs, V, H, DM, rho, prec);
    if (st != GINT_OK) return st;
    st = gint_batch_launch(b, stream);
    cudaError_t e = cudaStreamSynchronize(s);
    int w = 0;
    if (e == cudaSuccess) e = cudaMemcpy(&w, b->d_status, sizeof(int), cudaMemcpyDeviceToHost);
    gint_batch_destroy(b);
    if (st != GINT_OK) return st;
    if (e != cudaSuccess) return cuda_fail(e, "gint_batched");
    if (w != 0) {
        set_error("gint_batched: a kernel gave up on a bounded wait");
        return (gint_status)w;
    }
    return GINT_OK;
}

// ----------------------------------------------------------------------------- autotuner
extern "C" gint_status gint_autotune(const double cell[9], int natoms, const int *species, const double *tau,
                                     int nspecies, const gint_species *sp, const int grid[3], gint_prec prec,
                                     gint_options *best, double *ms_vlocal, double *ms_rho)
{
    if (!best || !tc_prec(prec)) {
        set_error("gint_autotune: need an output and a tensor-core precision");
        return GINT_EINVAL;
    }
    // vlocal shapes: at most 64 points, except for FP16x3, whose 16-deep MMA steps keep 128-point
    // batches inside the accumulation-error budget
    static const int cand_v32[][3] = {{4, 4, 4}, {4, 4, 2}, {2, 4, 4}, {4, 2, 4}, {2, 2, 8}, {8, 4, 2}};
    static const int cand_v16[][3] = {{4, 4, 8}, {4, 8, 4}, {8, 4, 4}, {4, 4, 4}, {4, 4, 6}, {2, 8, 8}};
    static const int cand_r[][3] = {{4, 4, 8}, {4, 8, 4}, {8, 4, 4}, {2, 8, 8}, {8, 8, 2}, {8, 2, 8}};
    const int(*cand_v)[3] = prec == GINT_FP16X3 ? cand_v16 : cand_v32;
    const int nc = 6;
    double bestv = 1e30, bestr = 1e30;
    gint_options o{};
    double *buf = nullptr;
    cudaEvent_t e0 = nullptr, e1 = nullptr;
    cudaError_t e = cudaEventCreate(&e0);
    if (e == cudaSuccess) e = cudaEventCreate(&e1);
    if (e != cudaSuccess) return cuda_fail(e, "gint_autotune");
    gint_status st = GINT_OK;
    size_t bufsz = 0;
    for (int c = 0; c < nc && st == GINT_OK; ++c) {
        gint_options opt{};
        for (int i = 0; i < 3; ++i) {
            opt.batch[i] = cand_v[c][i];
            opt.batch_rho[i] = cand_r[c][i];
        }
        gint_handle h = nullptr;
        if ((st = gint_setup(&h, cell, natoms, species, tau, nspecies, sp, grid, &opt)) != GINT_OK) break;
        const size_t np = (size_t)h->info.npts, nv = (size_t)h->info.nvalues;
        const size_t need = sizeof(double) * (2 * np + 2 * nv);
        if (need > bufsz) {
            if (buf) cudaFree(buf);
            if ((e = cudaMalloc((void **)&buf, need)) != cudaSuccess) {
                gint_destroy(h);
                st = cuda_fail(e, "gint_autotune: allocate");
                break;
            }
            bufsz = need;
            // synthetic inputs of the right sign structure; time does not depend on the values
            cudaMemset(buf, 0, need);
        }
        double *Vd = buf, *rhod = buf + np, *DMd = rhod + np, *Hd = DMd + nv;
        float tv = 0, tr = 0;
        for (int rep = 0; rep < 3 && st == GINT_OK; ++rep) {
            cudaEventRecord(e0, 0);
            st = gint_vlocal(h, Vd, Hd, prec, nullptr);
            cudaEventRecord(e1, 0);
            cudaEventSynchronize(e1);
            float t;
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) tv += t;
            cudaEventRecord(e0, 0);
            if (st == GINT_OK) st = gint_rho(h, DMd, rhod, prec, nullptr);
            cudaEventRecord(e1, 0);
            cudaEventSynchronize(e1);
            cudaEventElapsedTime(&t, e0, e1);
            if (rep > 0) tr += t;
        }
        gint_destroy(h);
        if (tv / 2 < bestv) {
            bestv = tv / 2;
            for (int i = 0; i < 3; ++i) o.batch[i] = cand_v[c][i];
        }
        if (tr / 2 < bestr) {
            bestr = tr / 2;
            for (int i = 0; i < 3; ++i) o.batch_rho[i] = cand_r[c][i];
        }
    }
    if (buf) cudaFree(buf);
    cudaEventDestroy(e0);
    cudaEventDestroy(e1);
    if (st != GINT_OK) return st;
    *best = o;
    if (ms_vlocal) *ms_vlocal = bestv;
    if (ms_rho) *ms_rho = bestr;
    return GINT_OK;
}
