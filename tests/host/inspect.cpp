// Test-only views of a handle's host arrays: compare two handles (a position update against a
// fresh set-up at the same positions), and read a decomposition's summary.
#include <cmath>
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
