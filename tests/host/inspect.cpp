// Test-only views of a handle's host arrays: compare two handles (a position update against a
// fresh set-up at the same positions), and read a decomposition's summary.
#include <array>
#include <cmath>
#include <map>
#include <cstdio>
#include <cstring>

#include "gint_internal.h"

using namespace gint;

template <class V>
static bool same_bytes(const V &a, const V &b)
{
    return a.size() == b.size() && (a.empty() || !memcmp(a.data(), b.data(), a.size() * sizeof(a[0])));
}

// 0 if equal; otherwise a bit per differing array (printed to stderr).  Slot positions are
// compared to 1e-12 bohr, everything else exactly.
extern "C" int inspect_compare(gint_handle a, gint_handle b)
{
    int bad = 0;
    for (int w = 0; w < 2; ++w) {
        const BatchSet &x = a->bs[w], &y = b->bs[w];
        const int sh = 10 * w;
        if (!same_bytes(x.batches, y.batches)) bad |= 1 << sh;
        if (!same_bytes(x.tbl, y.tbl)) bad |= 2 << sh;
        if (!same_bytes(x.tbl2, y.tbl2)) bad |= 4 << sh;
        if (!same_bytes(x.koff, y.koff)) bad |= 8 << sh;
        if (!same_bytes(x.slot_img, y.slot_img)) bad |= 16 << sh;
        if (x.slots.size() != y.slots.size()) {
            bad |= 32 << sh;
        } else {
            for (size_t i = 0; i < x.slots.size(); ++i) {
                const Slot &p = x.slots[i], &q = y.slots[i];
                bool d = p.atom != q.atom || p.species != q.species || p.orb_off != q.orb_off || p.norb != q.norb;
                for (int c = 0; c < 3; ++c) d = d || std::fabs(p.d0[c] - q.d0[c]) > 1e-12;
                if (d) {
                    bad |= 64 << sh;
                    break;
                }
            }
        }
        if (x.max_nb != y.max_nb || x.max_slots != y.max_slots || x.max_k != y.max_k || x.padn != y.padn ||
            std::fabs(x.flops_dense - y.flops_dense) > 1e-12 * std::fabs(y.flops_dense))
            bad |= 128 << sh;
    }
    if (a->keys != b->keys || a->offsets != b->offsets || a->partner != b->partner || a->soff != b->soff ||
        a->canon != b->canon || a->dms_plane != b->dms_plane)
        bad |= 1 << 20;
    if (bad) fprintf(stderr, "inspect_compare: difference mask 0x%x\n", bad);
    return bad;
}

// out[0..5] for decomposition w: batches, slots, table entries, padded layout, shared lists,
// largest padded width
extern "C" void inspect_summary(gint_handle a, int w, long long *out)
{
    const BatchSet &x = a->bs[w];
    out[0] = (long long)x.batches.size();
    out[1] = (long long)x.slots.size();
    out[2] = (long long)x.tbl.size();
    out[3] = x.padn;
    out[4] = x.shared;
    out[5] = x.max_k;
}

// Every slot-pair entry against the block list, looked up here through an ordered map of the
// block keys: tbl at tbl_index(a, b, ns) holds offset << 1 | canonical of block
// (I_a, I_b, n_b - n_a), or -1 if there is none, and the rho/force tbl2 (row-major) its
// split-store offset.  Returns the number of wrong entries.
extern "C" long long inspect_check_tables(gint_handle h)
{
    std::map<std::array<int, 5>, int> blk;
    const int64_t nblocks = (int64_t)h->keys.size() / 5;
    for (int64_t b = 0; b < nblocks; ++b) {
        const int32_t *k = &h->keys[5 * b];
        blk[{k[0], k[1], k[2], k[3], k[4]}] = (int)b;
    }
    long long bad = 0;
    for (int w = 0; w < 2; ++w) {
        const BatchSet &s = h->bs[w];
        for (const Batch &B : s.batches) {
            const int ns = B.nslots;
            for (int a = 0; a < ns; ++a)
                for (int b = 0; b < ns; ++b) {
                    const size_t sa = (size_t)B.slot0 + a, sb = (size_t)B.slot0 + b;
                    const int *na = &s.slot_img[3 * sa], *nb = &s.slot_img[3 * sb];
                    auto it = blk.find({s.slots[sa].atom, s.slots[sb].atom, nb[0] - na[0], nb[1] - na[1], nb[2] - na[2]});
                    const int bi = it == blk.end() ? -1 : it->second;
                    int want = -1;
                    if (bi >= 0) {
                        const int32_t *k = &h->keys[5 * bi];
                        auto pt = blk.find({k[1], k[0], -k[2], -k[3], -k[4]});
                        const bool canon = pt != blk.end() && bi <= pt->second;
                        want = (int)((h->offsets[bi] << 1) | (canon ? 1 : 0));
                    }
                    if (s.tbl[(size_t)B.tbl + tbl_index(a, b, ns)] != want) ++bad;
                    if (w == 1 && s.tbl2[(size_t)B.tbl + (size_t)a * ns + b] != (bi < 0 ? -1 : h->soff[bi])) ++bad;
                }
        }
    }
    return bad;
}

namespace gint {
std::vector<int2> segment_ranges(const Batch *b, const std::vector<int> &seg, int npart, int kind);
}

// Batches of decomposition w: out[4 i .. 4 i + 3] = points, orbitals, slots, first slot.
extern "C" long long inspect_batches(gint_handle h, int w, int *out, long long cap)
{
    const BatchSet &s = h->bs[w];
    const long long n = (long long)s.batches.size();
    for (long long i = 0; i < n && 4 * i + 3 < cap; ++i) {
        const Batch &B = s.batches[i];
        out[4 * i] = (B.dims & 255) * ((B.dims >> 8) & 255) * ((B.dims >> 16) & 255);
        out[4 * i + 1] = B.nb;
        out[4 * i + 2] = B.nslots;
        out[4 * i + 3] = B.slot0;
    }
    return n;
}

// The persistent kernels' CTA ranges for the batches of decomposition w cut into the segments
// seg[0..nseg]: out[2 (g npart + c)] = first, last + 1 of CTA c in segment g.
extern "C" void inspect_segment_ranges(gint_handle h, int w, const int *seg, int nseg, int npart, int *out)
{
    const std::vector<int> sv(seg, seg + nseg + 1);
    const std::vector<int2> r = segment_ranges(h->bs[w].batches.data(), sv, npart, w);
    for (size_t i = 0; i < r.size(); ++i) {
        out[2 * i] = r[i].x;
        out[2 * i + 1] = r[i].y;
    }
}
