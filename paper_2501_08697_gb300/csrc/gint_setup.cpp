// Host-side set-up of libgint: validation, radial splines, the block list (HContainer
// layout), grid batches and their atom-image lists, per-batch block tables, device upload.
//
// Paper references: NAO basis and strict locality (Sec. IV.A); block list over "all valid
// neighbouring cells" R and the HContainer store of H(R)/DM(R) (Sec. IV.B, Fig. 2 caption);
// grid partitioned into pieces that are integrated independently (Sec. IV.B).
#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <mutex>
#include <numeric>
#include <thread>
#include <unordered_map>

#include "gint_internal.h"

namespace gint {

static thread_local std::string g_err;

void set_error(const char *fmt, ...)
{
    char buf[1024];
    va_list ap;
    va_start(ap, fmt);
    vsnprintf(buf, sizeof(buf), fmt, ap);
    va_end(ap);
    g_err = buf;
}

const char *last_error() { return g_err.c_str(); }

gint_status cuda_fail(cudaError_t e, const char *where)
{
    set_error("%s: CUDA error %d (%s)", where, (int)e, cudaGetErrorString(e));
    return GINT_ECUDA;
}

// ---------------------------------------------------------------------------------------
// Clamped cubic spline in slope form: knot slopes k_i from
//   k_{i-1} + 4 k_i + k_{i+1} = 3 (y_{i+1} - y_{i-1}) / h,   k_0 = d0, k_{n-1} = dn,
// then each interval as a cubic in t = (r - r_i)/h in [0, 1).
static void spline_slopes(const double *y, int n, double h, double d0, double dn, std::vector<double> &k)
{
    k.assign(n, 0.0);
    k[0] = d0;
    k[n - 1] = dn;
    if (n <= 2) return;
    int m = n - 2;  // unknowns k_1 .. k_{n-2}
    std::vector<double> cp(m), dp(m);
    for (int j = 0; j < m; ++j) {
        int i = j + 1;
        double rhs = 3.0 * (y[i + 1] - y[i - 1]) / h;
        if (j == 0) rhs -= d0;
        if (j == m - 1) rhs -= dn;
        double diag = 4.0, lower = (j > 0) ? 1.0 : 0.0, upper = (j < m - 1) ? 1.0 : 0.0;
        double den = diag - (j > 0 ? lower * cp[j - 1] : 0.0);
        cp[j] = upper / den;
        dp[j] = (rhs - (j > 0 ? lower * dp[j - 1] : 0.0)) / den;
    }
    for (int j = m - 1; j >= 0; --j) k[j + 1] = dp[j] - (j < m - 1 ? cp[j] * k[j + 2] : 0.0);
}

static inline int64_t pack_key(int I, int J, int n1, int n2, int n3)
{
    return ((int64_t)I << 41) | ((int64_t)J << 21) | ((int64_t)(n1 + 64) << 14) | ((int64_t)(n2 + 64) << 7) |
           (int64_t)(n3 + 64);
}

struct Geo {
    double A[9];     // rows a_i
    double g[9];     // g[3*c + i]: component c of reciprocal vector g_i
    double gn[3];
    double det;
};

static Geo make_geo(const double *cell)
{
    Geo G;
    memcpy(G.A, cell, sizeof(G.A));
    const double *A = cell;
    G.det = A[0] * (A[4] * A[8] - A[5] * A[7]) - A[1] * (A[3] * A[8] - A[5] * A[6]) + A[2] * (A[3] * A[7] - A[4] * A[6]);
    for (int i = 0; i < 3; ++i) {
        const double *aj = A + 3 * ((i + 1) % 3), *ak = A + 3 * ((i + 2) % 3);
        double v[3] = {aj[1] * ak[2] - aj[2] * ak[1], aj[2] * ak[0] - aj[0] * ak[2], aj[0] * ak[1] - aj[1] * ak[0]};
        for (int c = 0; c < 3; ++c) G.g[3 * c + i] = v[c] / G.det;
        G.gn[i] = std::sqrt(v[0] * v[0] + v[1] * v[1] + v[2] * v[2]) / std::fabs(G.det);
    }
    return G;
}

static inline double frac_of(const Geo &G, const double *x, int i)
{
    return x[0] * G.g[0 + i] + x[1] * G.g[3 + i] + x[2] * G.g[6 + i];
}

// distance^2 from point c to the axis-aligned box [lo, hi] (orthogonal cells)
static inline double box_dist2(const double *c, const double *lo, const double *hi)
{
    double s = 0.0;
    for (int x = 0; x < 3; ++x) {
        double d = 0.0;
        if (c[x] < lo[x]) d = lo[x] - c[x];
        else if (c[x] > hi[x]) d = c[x] - hi[x];
        s += d * d;
    }
    return s;
}

struct RawSlot {
    int atom, n[3];
};

// Does the sphere (centre c, radius rc) touch any point of the batch box?  For orthogonal
// cells the exact box distance; otherwise a conservative centre-distance test.
struct BatchGeom {
    bool ortho;
    double h[9];  // a_i / N_i
};

static void batch_box(const BatchGeom &bg, int i0, int j0, int k0, int n1, int n2, int n3, double *lo, double *hi,
                      double *ctr, double *rad)
{
    // corners of the point parallelepiped
    double o[3], e[3][3];
    for (int c = 0; c < 3; ++c) {
        o[c] = i0 * bg.h[c] + j0 * bg.h[3 + c] + k0 * bg.h[6 + c];
        e[0][c] = (n1 - 1) * bg.h[c];
        e[1][c] = (n2 - 1) * bg.h[3 + c];
        e[2][c] = (n3 - 1) * bg.h[6 + c];
    }
    for (int c = 0; c < 3; ++c) {
        lo[c] = o[c] + std::min(0.0, e[0][c]) + std::min(0.0, e[1][c]) + std::min(0.0, e[2][c]);
        hi[c] = o[c] + std::max(0.0, e[0][c]) + std::max(0.0, e[1][c]) + std::max(0.0, e[2][c]);
        ctr[c] = o[c] + 0.5 * (e[0][c] + e[1][c] + e[2][c]);
    }
    double r2 = 0.0;
    for (int s1 = -1; s1 <= 1; s1 += 2)
        for (int s2 = -1; s2 <= 1; s2 += 2)
            for (int s3 = -1; s3 <= 1; s3 += 2) {
                double v[3];
                for (int c = 0; c < 3; ++c) v[c] = 0.5 * (s1 * e[0][c] + s2 * e[1][c] + s3 * e[2][c]);
                r2 = std::max(r2, v[0] * v[0] + v[1] * v[1] + v[2] * v[2]);
            }
    *rad = std::sqrt(r2);
}

static bool sphere_meets_batch(const BatchGeom &bg, const double *c, double rc, const double *lo, const double *hi,
                               const double *ctr, double rad)
{
    if (bg.ortho) return box_dist2(c, lo, hi) < rc * rc;
    double d[3] = {c[0] - ctr[0], c[1] - ctr[1], c[2] - ctr[2]};
    double dist = std::sqrt(d[0] * d[0] + d[1] * d[1] + d[2] * d[2]);
    return dist < rc + rad;
}

// ---------------------------------------------------------------------------------------
// Host threads for the set-up loops (the lists of different batches are independent).
static int host_threads()
{
    const unsigned n = std::thread::hardware_concurrency();
    return (int)std::max(1u, std::min(n, 64u));
}

// f(begin, end, part) over [0, n) split into contiguous parts, one host thread each; parts are
// numbered in index order so their outputs concatenate to the serial order.
template <class F>
static void parallel_parts(int64_t n, int nparts, F &&f)
{
    if (nparts <= 1 || n <= 1) {
        f((int64_t)0, n, 0);
        return;
    }
    std::vector<std::thread> th;
    th.reserve(nparts);
    for (int t = 0; t < nparts; ++t)
        th.emplace_back([&f, n, nparts, t] { f(n * t / nparts, n * (t + 1) / nparts, t); });
    for (auto &x : th) x.join();
}

// ---------------------------------------------------------------------------------------
// Position of a slot's atom image relative to its batch origin org: d0 = org - (tau_I + n.A),
// in FP64 and as an FP32 hi + lo pair.
static inline void slot_position(Slot &S, const double *org, const double *tau, const int *n, const Geo &G)
{
    for (int q = 0; q < 3; ++q) {
        S.d0[q] = org[q] - (tau[3 * S.atom + q] + n[0] * G.A[q] + n[1] * G.A[3 + q] + n[2] * G.A[6 + q]);
        S.dh[q] = (float)S.d0[q];
        S.dl[q] = (float)(S.d0[q] - (double)S.dh[q]);
    }
}

static inline void batch_origin(const BatchGeom &bg, int i0, int j0, int k0, double *org)
{
    for (int c = 0; c < 3; ++c) org[c] = i0 * bg.h[c] + j0 * bg.h[3 + c] + k0 * bg.h[6 + c];
}

// ---------------------------------------------------------------------------------------
// Batches of `out.dims` grid points, each with the atom images whose sphere meets it and the
// slot-pair -> block table; batches over the orbital or image limits are halved recursively.
// The base batches are processed in parts of consecutive a1 rows, one host thread each, and the
// parts concatenated in order (the result does not depend on the number of parts).
// With `old` (a position update): if every batch keeps its atom-image list, *same is set and
// out.slots receives old's slots at the new positions (nothing else of out is filled).
// Resizes a host array to n elements without initialising them; storage that must grow gets
// an eighth more, so that the next position updates (lists of about the same size, written
// into the storage this one replaces) need no new memory.
template <class V>
static void fit(V &v, size_t n)
{
    if (v.capacity() < n) {
        v.clear();
        v.reserve(n + n / 8);
    }
    v.resize(n);
}

// Accepted batches of one host thread's rows of top-level cells, in order, with their sorted
// atom-image lists.
struct BatchAcc {
    int i0, j0, k0, n1, n2, n3, r0, ns;   // accepted batch; its slots are raw[r0 .. r0 + ns)
};
struct BatchPart {
    std::vector<BatchAcc> acc;
    std::vector<RawSlot> raw;
    BatchSet s;
    gint_status st = GINT_OK;
    bool padfail = false;   // failed only because of the padded N width
    char err[256] = {0};
};

// The rho/force decomposition takes the vlocal lists when both use the same batch shape and
// limits and every vlocal batch fits the rho/force layout (its padded width, with the padded
// density layout): the vlocal build then also writes the rho/force slot-pair offsets.
struct ShareReq {
    const std::vector<int> *soff = nullptr;   // rho/force split-store offsets (null: no sharing)
    bool allow = false;                       // the lists may be shared (a position update keeps
                                              //   separate lists once the handle has them)
    bool padn = false;                        // rho/force layout is the padded one
    const BatchSet *old = nullptr;            // the handle's rho/force set, if it shared (update)
    hvec<int> *tbl2 = nullptr;                // out: rho/force slot-pair offsets
    bool ok = false;                          // out: the lists are shared
    std::vector<BatchPart> parts;             // out: the vlocal batches and lists, which seed the
                                              //   rho/force build when they are not shared
};

static gint_status build_batches(gint_handle h, const double *tau, const Geo &G, const BatchGeom &bg,
                                 const std::vector<double> &rc, const KeyIndex &kidx,
                                 const std::vector<int64_t> &offsets, const std::vector<uint8_t> &canon,
                                 const std::vector<int> &partner, const std::vector<int> *soff, ShareReq *share,
                                 const std::vector<BatchPart> *seed, bool padn, bool *pad_fail, const BatchSet *old,
                                 bool *same, BatchSet &out)
{
    const int natoms = h->natoms;
    const int N1 = h->grid[0], N2 = h->grid[1], N3 = h->grid[2];
    const int B1 = out.dims[0], B2 = out.dims[1], B3 = out.dims[2];
    const int nb1 = (N1 + B1 - 1) / B1, nb2 = (N2 + B2 - 1) / B2, nb3 = (N3 + B3 - 1) / B3;
    const int limit_nb = out.limit_nb;
    // padn (rho/force decomposition, padded density layout): the N axis is laid out like the
    // padded K axis, so the padded width must fit the accumulator's kMaxNb columns too
    if (same) *same = false;
    if (pad_fail) *pad_fail = false;
    using Acc = BatchAcc;
    using Part = BatchPart;
    const int nparts = std::min(host_threads(), nb1);
    std::vector<Part> parts(nparts);
    if (seed && (int)seed->size() != nparts) seed = nullptr;
    auto orb_count = [&](const std::vector<RawSlot> &s) {
        int n = 0;
        for (auto &x : s) n += h->norb_atom[x.atom];
        return n;
    };
    // padded K width of a slot list and, with koff, each slot's first padded column: slot widths
    // rounded up to kpad; slots of up to kKSeg columns do not cross a multiple of kKSeg, wider
    // ones start on one.  In the rho/force decomposition the same offsets are the N columns, so
    // a list whose segment-aligned width exceeds the accumulator's kMaxNb columns is packed
    // densely instead (the density kernel then evaluates a straddling slot once per segment).
    auto padded_width = [&](const RawSlot *s, int ns, std::vector<int> *koff) {
        const size_t k0 = koff ? koff->size() : 0;
        int kcur = 0;
        for (int i = 0; i < ns; ++i) {
            const int kw = kpad(h->norb_atom[s[i].atom]);
            if ((kw <= kKSeg && kcur % kKSeg + kw > kKSeg) || (kw > kKSeg && kcur % kKSeg))
                kcur = (kcur / kKSeg + 1) * kKSeg;
            if (koff) koff->push_back(kcur);
            kcur += kw;
        }
        if (padn && kcur > kMaxNb) {
            if (koff) koff->resize(k0);
            kcur = 0;
            for (int i = 0; i < ns; ++i) {
                if (koff) koff->push_back(kcur);
                kcur += kpad(h->norb_atom[s[i].atom]);
            }
        }
        return kcur;
    };
    // Atom images ordered by atom ascending, then image n descending.  With this order every
    // pair of slots a < b maps to the canonical member of its partner pair {(I,J,R), (J,I,-R)}:
    // I_a < I_b, or I_a == I_b with R = n_b - n_a lexicographically negative.  The tensor-core
    // scatter relies on it (it adds only elements with row <= column).
    auto slot_less = [](const RawSlot &a, const RawSlot &b) {
        if (a.atom != b.atom) return a.atom < b.atom;
        if (a.n[0] != b.n[0]) return a.n[0] > b.n[0];
        if (a.n[1] != b.n[1]) return a.n[1] > b.n[1];
        return a.n[2] > b.n[2];
    };
    // phase 1: the accepted batches and their sorted atom-image lists
    parallel_parts(nb1, nparts, [&](int64_t r0, int64_t r1, int part) {
        Part &pt = parts[part];
        auto fail = [&](const char *fmt, int x, int y) {
            if (pt.st == GINT_OK) {
                snprintf(pt.err, sizeof(pt.err), fmt, x, y);
                pt.st = GINT_EINVAL;
            }
        };
        struct Work {
            int i0, j0, k0, n1, n2, n3;
            std::vector<RawSlot> s;
        };
        // accepts w0, or splits it (halving the longest axis) until every piece fits the limits
        auto run = [&](Work &&w0) {
            std::vector<Work> stack;
            stack.push_back(std::move(w0));
            while (!stack.empty() && pt.st == GINT_OK) {
                Work w = std::move(stack.back());
                stack.pop_back();
                std::sort(w.s.begin(), w.s.end(), slot_less);
                int nb = orb_count(w.s);
                const int pw = padn ? padded_width(w.s.data(), (int)w.s.size(), nullptr) : 0;
                if (nb > limit_nb || (int)w.s.size() > kMaxSlots || pw > kMaxNb) {
                    // halve the longest axis; a3 halves stay even so batch origins stay even
                    int dims[3] = {w.n1, w.n2, w.n3};
                    int ax = -1;
                    for (int a = 0; a < 3; ++a) {
                        bool can = (a == 2) ? dims[a] >= 4 : dims[a] >= 2;
                        if (can && (ax < 0 || dims[a] > dims[ax])) ax = a;
                    }
                    if (ax < 0) {
                        // cannot split further: accept up to the hard kernel limits
                        if (nb <= kMaxNb && (int)w.s.size() <= kMaxSlots && pw <= kMaxNb) goto accept;
                        if (nb <= kMaxNb && (int)w.s.size() <= kMaxSlots) pt.padfail = true;
                        fail("gint_setup: a grid batch sees %d orbitals / %d atom images", nb, (int)w.s.size());
                        break;
                    }
                    int cut = dims[ax] / 2;
                    if (ax == 2 && (cut % 2)) cut += 1;
                    Work a = w, b = w;
                    if (ax == 0) { a.n1 = cut; b.i0 += cut; b.n1 -= cut; }
                    if (ax == 1) { a.n2 = cut; b.j0 += cut; b.n2 -= cut; }
                    if (ax == 2) { a.n3 = cut; b.k0 += cut; b.n3 -= cut; }
                    for (Work *x : {&b, &a}) {
                        double lo3[3], hi3[3], ctr[3], rad;
                        batch_box(bg, x->i0, x->j0, x->k0, x->n1, x->n2, x->n3, lo3, hi3, ctr, &rad);
                        std::vector<RawSlot> keep;
                        for (auto &s : w.s) {
                            double c[3];
                            for (int q = 0; q < 3; ++q)
                                c[q] = tau[3 * s.atom + q] + s.n[0] * G.A[q] + s.n[1] * G.A[3 + q] + s.n[2] * G.A[6 + q];
                            if (sphere_meets_batch(bg, c, rc[s.atom], lo3, hi3, ctr, rad)) keep.push_back(s);
                        }
                        x->s = std::move(keep);
                        stack.push_back(std::move(*x));
                    }
                    continue;
                }
            accept:
                pt.acc.push_back({w.i0, w.j0, w.k0, w.n1, w.n2, w.n3, (int)pt.raw.size(), (int)w.s.size()});
                pt.raw.insert(pt.raw.end(), w.s.begin(), w.s.end());
            }
        };
        if (seed) {
            // the vlocal batches of these rows (same shape and limits): this decomposition
            // splits them further where a batch exceeds the padded layout's width
            const Part &sp = (*seed)[part];
            pt.raw.reserve(sp.raw.size());
            pt.acc.reserve(sp.acc.size());
            for (const Acc &A : sp.acc) {
                if (pt.st != GINT_OK) break;
                const RawSlot *l = sp.raw.data() + A.r0;
                if (!padn || padded_width(l, A.ns, nullptr) <= kMaxNb) {
                    pt.acc.push_back({A.i0, A.j0, A.k0, A.n1, A.n2, A.n3, (int)pt.raw.size(), A.ns});
                    pt.raw.insert(pt.raw.end(), l, l + A.ns);
                } else {
                    run(Work{A.i0, A.j0, A.k0, A.n1, A.n2, A.n3, std::vector<RawSlot>(l, l + A.ns)});
                }
            }
            return;
        }
        const int rows = (int)(r1 - r0);
        std::vector<std::vector<RawSlot>> lists((size_t)rows * nb2 * nb3);
        for (auto &l : lists) l.reserve(32);
        for (int I = 0; I < natoms; ++I) {
            const double *t = tau + 3 * I;
            int lo[3], hi[3];
            for (int i = 0; i < 3; ++i) {
                double s = frac_of(G, t, i);
                lo[i] = (int)std::floor(-s - rc[I] * G.gn[i]) - 1;
                hi[i] = (int)std::ceil(1.0 - s + rc[I] * G.gn[i]) + 1;
            }
            for (int n1 = lo[0]; n1 <= hi[0]; ++n1)
                for (int n2 = lo[1]; n2 <= hi[1]; ++n2)
                    for (int n3 = lo[2]; n3 <= hi[2]; ++n3) {
                        double c[3];
                        for (int x = 0; x < 3; ++x) c[x] = t[x] + n1 * G.A[x] + n2 * G.A[3 + x] + n3 * G.A[6 + x];
                        int ilo[3], ihi[3];
                        bool empty = false;
                        for (int i = 0; i < 3; ++i) {
                            double s = frac_of(G, c, i) * h->grid[i];
                            double ext = rc[I] * G.gn[i] * h->grid[i];
                            ilo[i] = std::max(0, (int)std::floor(s - ext) - 1);
                            ihi[i] = std::min(h->grid[i] - 1, (int)std::ceil(s + ext) + 1);
                            if (ilo[i] > ihi[i]) empty = true;
                        }
                        if (empty) continue;
                        const int b1lo = std::max<int>(ilo[0] / B1, (int)r0), b1hi = std::min<int>(ihi[0] / B1, (int)r1 - 1);
                        const int b2lo = ilo[1] / B2, b2hi = ihi[1] / B2, b3lo = ilo[2] / B3, b3hi = ihi[2] / B3;
                        if (b1lo > b1hi) continue;
                        if (bg.ortho) {
                            // the box distance of an orthogonal cell separates by axis: the same
                            // sum as box_dist2, from per-row / column / layer squared distances
                            const double rr = rc[I] * rc[I];
                            auto d2 = [&](int ax, int b, int Bx, int Nx) {
                                const int i0 = b * Bx, np = std::min(Bx, Nx - i0);
                                const double o = i0 * bg.h[4 * ax], e = (np - 1) * bg.h[4 * ax];
                                const double lo = o + std::min(0.0, e), hi = o + std::max(0.0, e);
                                const double d = c[ax] < lo ? lo - c[ax] : (c[ax] > hi ? c[ax] - hi : 0.0);
                                return d * d;
                            };
                            double dz2[64];
                            const int n3c = std::min(b3hi - b3lo + 1, 64);
                            for (int q = 0; q < n3c; ++q) dz2[q] = d2(2, b3lo + q, B3, N3);
                            for (int b1 = b1lo; b1 <= b1hi; ++b1) {
                                const double s1 = 0.0 + d2(0, b1, B1, N1);
                                if (!(s1 < rr)) continue;
                                for (int b2 = b2lo; b2 <= b2hi; ++b2) {
                                    const double s12 = s1 + d2(1, b2, B2, N2);
                                    if (!(s12 < rr)) continue;
                                    for (int b3 = b3lo; b3 <= b3hi; ++b3) {
                                        const double dz = b3 - b3lo < 64 ? dz2[b3 - b3lo] : d2(2, b3, B3, N3);
                                        if (s12 + dz < rr)
                                            lists[((size_t)(b1 - r0) * nb2 + b2) * nb3 + b3].push_back({I, {n1, n2, n3}});
                                    }
                                }
                            }
                            continue;
                        }
                        for (int b1 = b1lo; b1 <= b1hi; ++b1)
                            for (int b2 = b2lo; b2 <= b2hi; ++b2)
                                for (int b3 = b3lo; b3 <= b3hi; ++b3) {
                                    int i0 = b1 * B1, j0 = b2 * B2, k0 = b3 * B3;
                                    int n1p = std::min(B1, N1 - i0), n2p = std::min(B2, N2 - j0), n3p = std::min(B3, N3 - k0);
                                    double lo3[3], hi3[3], ctr[3], rad;
                                    batch_box(bg, i0, j0, k0, n1p, n2p, n3p, lo3, hi3, ctr, &rad);
                                    if (sphere_meets_batch(bg, c, rc[I], lo3, hi3, ctr, rad))
                                        lists[((size_t)(b1 - r0) * nb2 + b2) * nb3 + b3].push_back({I, {n1, n2, n3}});
                                }
                    }
        }
        {
            size_t nraw = 0;
            for (const auto &l : lists) nraw += l.size();
            pt.raw.reserve(nraw);
            pt.acc.reserve(lists.size());
        }
        for (int b1 = (int)r0; b1 < (int)r1 && pt.st == GINT_OK; ++b1)
            for (int b2 = 0; b2 < nb2; ++b2)
                for (int b3 = 0; b3 < nb3; ++b3) {
                    std::vector<RawSlot> &l0 = lists[((size_t)(b1 - r0) * nb2 + b2) * nb3 + b3];
                    const int n01 = std::min(B1, N1 - b1 * B1), n02 = std::min(B2, N2 - b2 * B2),
                              n03 = std::min(B3, N3 - b3 * B3);
                    {
                        // the common case, a cell that needs no split, without the work stack
                        std::sort(l0.begin(), l0.end(), slot_less);
                        const int pw = padn ? padded_width(l0.data(), (int)l0.size(), nullptr) : 0;
                        if (orb_count(l0) <= limit_nb && (int)l0.size() <= kMaxSlots && pw <= kMaxNb) {
                            pt.acc.push_back({b1 * B1, b2 * B2, b3 * B3, n01, n02, n03, (int)pt.raw.size(), (int)l0.size()});
                            pt.raw.insert(pt.raw.end(), l0.begin(), l0.end());
                            continue;
                        }
                    }
                    run(Work{b1 * B1, b2 * B2, b3 * B3, n01, n02, n03, std::move(l0)});
                }
    });
    std::vector<size_t> bat0(nparts + 1, 0);
    for (int t = 0; t < nparts; ++t) {
        if (parts[t].st != GINT_OK) {
            set_error("%s", parts[t].err);
            if (pad_fail) *pad_fail = parts[t].padfail;
            return parts[t].st;
        }
        bat0[t + 1] = bat0[t] + parts[t].acc.size();
    }
    if (bat0[nparts] >= ((size_t)1 << 31)) {
        set_error("gint_setup: too many batches");
        return GINT_EINVAL;
    }
    if (share && share->soff) {
        std::vector<int> fits(nparts, 1);
        if (share->padn && share->allow)
            parallel_parts(nparts, nparts, [&](int64_t t0, int64_t t1, int) {
                for (int64_t t = t0; t < t1; ++t)
                    for (const Acc &A : parts[t].acc)
                        if (padded_width(parts[t].raw.data() + A.r0, A.ns, nullptr) > kMaxNb) {
                            fits[t] = 0;
                            break;
                        }
            });
        share->ok = share->allow && std::all_of(fits.begin(), fits.end(), [](int x) { return x != 0; });
    }
    // a position update whose lists are all unchanged: the old slots at the new positions
    if (old && old->batches.size() == bat0[nparts]) {
        std::vector<int> eq(nparts, 1);
        parallel_parts(nparts, nparts, [&](int64_t t0, int64_t t1, int) {
            for (int64_t t = t0; t < t1; ++t) {
                const Part &pt = parts[t];
                for (size_t q = 0; q < pt.acc.size() && eq[t]; ++q) {
                    const Acc &A = pt.acc[q];
                    const Batch &B = old->batches[bat0[t] + q];
                    if (B.i0 != A.i0 || B.j0 != A.j0 || B.k0 != A.k0 || B.dims != (A.n1 | (A.n2 << 8) | (A.n3 << 16)) ||
                        B.nslots != A.ns) {
                        eq[t] = 0;
                        break;
                    }
                    for (int s = 0; s < A.ns; ++s) {
                        const RawSlot &r = pt.raw[A.r0 + s];
                        const int *n = &old->slot_img[3 * ((size_t)B.slot0 + s)];
                        if (old->slots[B.slot0 + s].atom != r.atom || n[0] != r.n[0] || n[1] != r.n[1] || n[2] != r.n[2]) {
                            eq[t] = 0;
                            break;
                        }
                    }
                }
            }
        });
        if (std::all_of(eq.begin(), eq.end(), [](int x) { return x != 0; })) {
            // the caller writes the new slot positions into the handle's records
            if (same) *same = true;
            if (share && share->soff) share->parts = std::move(parts);
            return GINT_OK;
        }
    }
    // phase 2: slot records, padded K offsets and slot-pair block tables, written in place (the
    // parts' offsets are known from phase 1).  A batch whose origin, shape and atom-image list
    // equal those of a batch of `old` copies its tables and offsets from there and only gets new
    // slot positions; the others look their blocks up.
    std::vector<size_t> sl0(nparts + 1, 0), tb0(nparts + 1, 0);
    for (int t = 0; t < nparts; ++t) {
        size_t ns = 0, nt = 0;
        for (const Acc &A : parts[t].acc) {
            ns += A.ns;
            nt += (size_t)A.ns * A.ns;
        }
        sl0[t + 1] = sl0[t] + ns;
        tb0[t + 1] = tb0[t] + nt;
    }
    if ((int64_t)tb0[nparts] >= ((int64_t)1 << 31) || sl0[nparts] >= ((size_t)1 << 31)) {
        set_error("gint_setup: too many batches / table entries");
        return GINT_EINVAL;
    }
    fit(out.batches, bat0[nparts]);
    fit(out.slots, sl0[nparts]);
    fit(out.slot_img, 3 * sl0[nparts]);
    fit(out.koff, sl0[nparts]);
    fit(out.tbl, tb0[nparts]);
    // slot-pair offsets into the split store: this set's own (rho/force), or the rho/force set's
    // when it shares these lists (written next to the vlocal tables)
    const std::vector<int> *sf = soff ? soff : (share && share->ok ? share->soff : nullptr);
    hvec<int> *t2v = soff ? &out.tbl2 : (sf ? share->tbl2 : nullptr);
    if (t2v) fit(*t2v, tb0[nparts]);
    int *const t2 = t2v ? t2v->data() : nullptr;
    const hvec<int> *old_t2 = !old ? nullptr : soff ? &old->tbl2 : (sf && share->old ? &share->old->tbl2 : nullptr);
    // batches of old by top-level cell: the batches a cell was split into are consecutive
    // (cell -> first such batch, or -1)
    const bool reuse =
        old && old->koff.size() == old->slots.size() && (!sf || (old_t2 && old_t2->size() == old->tbl.size()));
    std::vector<int> oldcell;
    auto cell_of = [&](int i0, int j0, int k0) { return ((int64_t)(i0 / B1) * nb2 + j0 / B2) * nb3 + k0 / B3; };
    if (reuse) {
        oldcell.assign((size_t)nb1 * nb2 * nb3, -1);
        for (size_t q = old->batches.size(); q-- > 0;) {
            const Batch &B = old->batches[q];
            oldcell[cell_of(B.i0, B.j0, B.k0)] = (int)q;
        }
    }
    parallel_parts(nparts, nparts, [&](int64_t t0, int64_t t1, int) {
        for (int64_t t = t0; t < t1; ++t) {
            Part &pt = parts[t];
            BatchSet &o = pt.s;   // per-part statistics only
            size_t so = sl0[t], to = tb0[t];
            for (size_t q = 0; q < pt.acc.size() && pt.st == GINT_OK; ++q) {
                const Acc &A = pt.acc[q];
                const RawSlot *ws = pt.raw.data() + A.r0;
                int nb = 0;
                for (int s = 0; s < A.ns; ++s) nb += h->norb_atom[ws[s].atom];
                Batch B{};
                B.i0 = A.i0; B.j0 = A.j0; B.k0 = A.k0;
                B.dims = A.n1 | (A.n2 << 8) | (A.n3 << 16);
                B.slot0 = (int)so;
                B.nslots = A.ns;
                B.nb = nb;
                B.tbl = (int)to;
                o.flops_dense += 2.0 * (A.n1 * A.n2 * A.n3) * (double)nb * nb;
                o.max_nb = std::max(o.max_nb, nb);
                o.max_slots = std::max(o.max_slots, A.ns);
                double org[3];
                batch_origin(bg, A.i0, A.j0, A.k0, org);
                const Batch *ob = nullptr, *near = nullptr;   // old batch at this origin: same list / other
                if (reuse) {
                    const int64_t cell = cell_of(A.i0, A.j0, A.k0);
                    int q0 = oldcell[cell];
                    while (q0 >= 0 && q0 < (int)old->batches.size() &&
                           cell_of(old->batches[q0].i0, old->batches[q0].j0, old->batches[q0].k0) == cell &&
                           (old->batches[q0].i0 != A.i0 || old->batches[q0].j0 != A.j0 || old->batches[q0].k0 != A.k0))
                        ++q0;
                    if (q0 >= 0 && q0 < (int)old->batches.size() && old->batches[q0].i0 == A.i0 &&
                        old->batches[q0].j0 == A.j0 && old->batches[q0].k0 == A.k0) {
                        const Batch &C = old->batches[q0];
                        bool eq = C.dims == B.dims && C.nslots == A.ns;
                        for (int s = 0; eq && s < A.ns; ++s) {
                            const int *n = &old->slot_img[3 * ((size_t)C.slot0 + s)];
                            eq = old->slots[C.slot0 + s].atom == ws[s].atom && n[0] == ws[s].n[0] && n[1] == ws[s].n[1] &&
                                 n[2] == ws[s].n[2];
                        }
                        if (eq) ob = &C;
                        else near = &C;
                    }
                }
                if (ob) {
                    // unchanged list: the old records at the new positions, the old tables
                    for (int s = 0; s < A.ns; ++s) {
                        Slot S = old->slots[ob->slot0 + s];
                        slot_position(S, org, tau, ws[s].n, G);
                        out.slots[so + s] = S;
                        out.koff[so + s] = old->koff[ob->slot0 + s];
                    }
                    std::copy_n(old->slot_img.begin() + 3 * (size_t)ob->slot0, 3 * A.ns, out.slot_img.begin() + 3 * so);
                    std::copy_n(old->tbl.begin() + ob->tbl, (size_t)A.ns * A.ns, out.tbl.begin() + to);
                    if (t2) std::copy_n(old_t2->begin() + ob->tbl, (size_t)A.ns * A.ns, t2 + to);
                    o.max_k = std::max(o.max_k, padded_width(ws, A.ns, nullptr));
                } else {
                    std::vector<int> ko;
                    ko.reserve(A.ns);
                    o.max_k = std::max(o.max_k, padded_width(ws, A.ns, &ko));
                    int off = 0;
                    for (int s = 0; s < A.ns; ++s) {
                        Slot S{};
                        S.atom = ws[s].atom;
                        S.species = h->species[ws[s].atom];
                        S.orb_off = off;
                        S.norb = h->norb_atom[ws[s].atom];
                        slot_position(S, org, tau, ws[s].n, G);
                        off += S.norb;
                        out.slots[so + s] = S;
                        out.koff[so + s] = ko[s];
                        for (int c = 0; c < 3; ++c) out.slot_img[3 * (so + s) + c] = ws[s].n[c];
                    }
                    // om[s]: the slot of the old batch at this origin with the same atom image, or
                    // -1 (both lists are in slot order); a pair of such slots takes the old entries
                    int om[kMaxSlots];
                    for (int s = 0; s < A.ns; ++s) om[s] = -1;
                    if (near)
                        for (int s = 0, j = 0; s < A.ns && j < near->nslots;) {
                            const size_t g = (size_t)near->slot0 + j;
                            const RawSlot r{old->slots[g].atom,
                                            {old->slot_img[3 * g], old->slot_img[3 * g + 1], old->slot_img[3 * g + 2]}};
                            if (slot_less(ws[s], r)) {
                                ++s;
                            } else if (slot_less(r, ws[s])) {
                                ++j;
                            } else {
                                om[s++] = j++;
                            }
                        }
                    // one look-up per unordered slot pair: block (I_b, I_a, n_a - n_b) of the pair
                    // (b, a) is the partner of block (I_a, I_b, n_b - n_a)
                    for (int ia = 0; ia < A.ns && pt.st == GINT_OK; ++ia)
                        for (int ib = ia; ib < A.ns; ++ib) {
                            // x, xt: entries of (a, b) and (b, a) in the vlocal table layout
                            // (tbl_index), y, yt: in the row-major split-store table
                            const size_t x = to + tbl_index(ia, ib, A.ns), xt = to + tbl_index(ib, ia, A.ns);
                            const size_t y = to + (size_t)ia * A.ns + ib, yt = to + (size_t)ib * A.ns + ia;
                            if (om[ia] >= 0 && om[ib] >= 0) {
                                const int na = near->nslots, a0 = om[ia], b0 = om[ib];
                                out.tbl[x] = old->tbl[(size_t)near->tbl + tbl_index(a0, b0, na)];
                                out.tbl[xt] = old->tbl[(size_t)near->tbl + tbl_index(b0, a0, na)];
                                if (t2) {
                                    t2[y] = (*old_t2)[(size_t)near->tbl + (size_t)a0 * na + b0];
                                    t2[yt] = (*old_t2)[(size_t)near->tbl + (size_t)b0 * na + a0];
                                }
                                continue;
                            }
                            const RawSlot &sa = ws[ia], &sb = ws[ib];
                            const int bi = kidx.find(
                                pack_key(sa.atom, sb.atom, sb.n[0] - sa.n[0], sb.n[1] - sa.n[1], sb.n[2] - sa.n[2]));
                            if (bi < 0) {
                                out.tbl[x] = out.tbl[xt] = -1;
                                if (t2) t2[y] = t2[yt] = -1;
                                continue;
                            }
                            if (!canon[bi]) {
                                snprintf(pt.err, sizeof(pt.err), "%s",
                                         "gint_setup: internal error, slot order breaks the canonical-pair rule");
                                pt.st = GINT_EINVAL;
                                break;
                            }
                            const int bt = partner[bi];
                            out.tbl[x] = (int)((offsets[bi] << 1) | canon[bi]);
                            out.tbl[xt] = (int)((offsets[bt] << 1) | canon[bt]);
                            if (t2) {
                                t2[y] = (*sf)[bi];
                                t2[yt] = (*sf)[bt];
                            }
                        }
                }
                out.batches[bat0[t] + q] = B;
                so += A.ns;
                to += (size_t)A.ns * A.ns;
            }
            if (!(share && share->soff)) std::vector<RawSlot>().swap(pt.raw);
        }
    });
    for (auto &pt : parts) {
        if (pt.st != GINT_OK) {
            set_error("%s", pt.err);
            return pt.st;
        }
        out.flops_dense += pt.s.flops_dense;
        out.max_nb = std::max(out.max_nb, pt.s.max_nb);
        out.max_slots = std::max(out.max_slots, pt.s.max_slots);
        out.max_k = std::max(out.max_k, pt.s.max_k);
    }
    if (share && share->soff) share->parts = std::move(parts);
    return GINT_OK;
}

static BatchGeom batch_geom(const gint_handle_s *h)
{
    BatchGeom bg;
    bg.ortho = true;
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c)
            if (i != c && h->cell[3 * i + c] != 0.0) bg.ortho = false;
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) bg.h[3 * i + c] = h->cell[3 * i + c] / h->grid[i];
    return bg;
}

template <class V>
static void par_copy(V &dst, const V &src)
{
    fit(dst, src.size());
    parallel_parts((int64_t)src.size(), src.size() < ((size_t)1 << 16) ? 1 : host_threads(),
                   [&](int64_t a, int64_t b, int) { std::copy(src.begin() + a, src.begin() + b, dst.begin() + a); });
}

// Moves the host arrays of src into dst, emptied but keeping their capacity.
static void take_storage(BatchSet &dst, BatchSet &src)
{
    dst.batches = std::move(src.batches);
    dst.slots = std::move(src.slots);
    dst.slot_img = std::move(src.slot_img);
    dst.tbl = std::move(src.tbl);
    dst.koff = std::move(src.koff);
    dst.tbl2 = std::move(src.tbl2);
    for (auto *v : {&dst.slot_img, &dst.tbl, &dst.koff, &dst.tbl2}) v->clear();
    dst.batches.clear();
    dst.slots.clear();
}

// New positions of the slots of a decomposition whose atom-image lists are unchanged, in place.
static void place_slots(const gint_handle_s *h, BatchSet &bs, const double *tau)
{
    const Geo G = make_geo(h->cell);
    const BatchGeom bg = batch_geom(h);
    parallel_parts((int64_t)bs.batches.size(), host_threads(), [&](int64_t q0, int64_t q1, int) {
        for (int64_t q = q0; q < q1; ++q) {
            const Batch &B = bs.batches[q];
            double org[3];
            batch_origin(bg, B.i0, B.j0, B.k0, org);
            for (int s = 0; s < B.nslots; ++s)
                slot_position(bs.slots[B.slot0 + s], org, tau, &bs.slot_img[3 * ((size_t)B.slot0 + s)], G);
        }
    });
}

// ---------------------------------------------------------------------------------------
gint_status build_geometry(gint_handle h, const double *tau, const gint_handle_s *old)
{
    const bool update_only = old != nullptr;
    const int natoms = h->natoms;
    Geo G = make_geo(h->cell);
    Plan &P = h->plan;
    const int N1 = h->grid[0], N2 = h->grid[1], N3 = h->grid[2];
    std::vector<double> rc(natoms);
    for (int I = 0; I < natoms; ++I) rc[I] = P.sp[h->species[I]].rcut;

    // ---- block list: all (I, J, n) with |tau_J + n.A - tau_I| < rc_I + rc_J (rows I in parts,
    // one host thread each, joined in order).  |v| < r bounds the fractional coordinate
    // g_i.v = s_i + n_i of v by r |g_i|, which gives each image index's range.
    std::vector<int32_t> keys;
    std::vector<int64_t> packed;
    {
        std::vector<double> fr(3 * (size_t)natoms);
        for (int I = 0; I < natoms; ++I)
            for (int i = 0; i < 3; ++i) fr[3 * I + i] = frac_of(G, tau + 3 * I, i);
        const int nparts = std::min(host_threads(), natoms);
        std::vector<std::vector<int32_t>> pkeys(nparts);
        std::vector<std::vector<int64_t>> ppacked(nparts);
        std::vector<int> bad(nparts, 0);
        parallel_parts(natoms, nparts, [&](int64_t i0, int64_t i1, int part) {
            for (int I = (int)i0; I < (int)i1 && !bad[part]; ++I) {
                for (int J = 0; J < natoms; ++J) {
                    const double rs = rc[I] + rc[J], rr = rs * rs;
                    const double dt[3] = {tau[3 * J] - tau[3 * I], tau[3 * J + 1] - tau[3 * I + 1],
                                          tau[3 * J + 2] - tau[3 * I + 2]};
                    int lo[3], hi[3];
                    for (int i = 0; i < 3; ++i) {
                        const double s = fr[3 * J + i] - fr[3 * I + i], x = rs * G.gn[i];
                        lo[i] = (int)std::floor(-s - x);
                        hi[i] = (int)std::ceil(-s + x);
                    }
                    for (int n1 = lo[0]; n1 <= hi[0]; ++n1)
                        for (int n2 = lo[1]; n2 <= hi[1]; ++n2) {
                            double v12[3];
                            for (int x = 0; x < 3; ++x) v12[x] = dt[x] + n1 * G.A[x] + n2 * G.A[3 + x];
                            for (int n3 = lo[2]; n3 <= hi[2]; ++n3) {
                                const double v[3] = {v12[0] + n3 * G.A[6], v12[1] + n3 * G.A[7], v12[2] + n3 * G.A[8]};
                                if (v[0] * v[0] + v[1] * v[1] + v[2] * v[2] < rr) {
                                    if (std::abs(n1) > 63 || std::abs(n2) > 63 || std::abs(n3) > 63) bad[part] = 1;
                                    pkeys[part].insert(pkeys[part].end(), {I, J, n1, n2, n3});
                                    if (!update_only) ppacked[part].push_back(pack_key(I, J, n1, n2, n3));
                                }
                            }
                        }
                }
            }
        });
        for (int t = 0; t < nparts; ++t) {
            if (bad[t]) {
                set_error("gint_setup: periodic image index beyond 63 (cell too small for rcut)");
                return GINT_EINVAL;
            }
        }
        if (update_only) {
            // the block list must be the handle's, in the same order
            bool eq = true;
            size_t at = 0;
            for (int t = 0; t < nparts && eq; ++t) {
                eq = at + pkeys[t].size() <= old->keys.size() &&
                     std::equal(pkeys[t].begin(), pkeys[t].end(), old->keys.begin() + at);
                at += pkeys[t].size();
            }
            if (!eq || at != old->keys.size()) {
                set_error("gint_update_positions: block list changed; build a new handle");
                return GINT_ESTATE;
            }
        } else {
            for (int t = 0; t < nparts; ++t) {
                keys.insert(keys.end(), pkeys[t].begin(), pkeys[t].end());
                packed.insert(packed.end(), ppacked[t].begin(), ppacked[t].end());
            }
        }
    }
    // Block offsets, split-store offsets, key index and partner blocks depend on the block list
    // only: a position update (same list) takes the handle's.
    std::vector<int64_t> offsets;
    std::vector<int> soff_pad, soff_row, partner;
    std::vector<uint8_t> canon;
    KeyIndex kidx_new;
    int64_t splane_pad = 0, splane_row = 0;
    if (!update_only) {
        const int64_t nblocks = (int64_t)packed.size();
        offsets.assign(nblocks + 1, 0);
        for (int64_t b = 0; b < nblocks; ++b)
            offsets[b + 1] = offsets[b] + (int64_t)h->norb_atom[keys[5 * b]] * h->norb_atom[keys[5 * b + 1]];
        if (offsets[nblocks] >= ((int64_t)1 << 30)) {
            set_error("gint_setup: block store of %lld values exceeds 2^30", (long long)offsets[nblocks]);
            return GINT_EINVAL;
        }
        // offsets of the blocks in the split density-matrix store, per term.  Padded layout: rows
        // and columns padded to kpad, a block holds all its terms (element offset NT soff[b]).
        // Row layout: rows n_I, columns padded, each term in its own plane of splane elements.
        soff_pad.resize(nblocks);
        soff_row.resize(nblocks);
        for (int64_t b = 0; b < nblocks; ++b) {
            const int nI = h->norb_atom[keys[5 * b]], nJ = h->norb_atom[keys[5 * b + 1]];
            soff_pad[b] = (int)splane_pad;
            soff_row[b] = (int)splane_row;
            splane_pad += (int64_t)kpad(nI) * kpad(nJ);
            splane_row += (int64_t)nI * kpad(nJ);
        }
        if (splane_pad >= ((int64_t)1 << 30)) {   // the larger of the two
            set_error("gint_setup: padded block store of %lld values exceeds 2^30", (long long)splane_pad);
            return GINT_EINVAL;
        }
        kidx_new = KeyIndex(packed);
        partner.resize(nblocks);
        canon.resize(nblocks);
        for (int64_t b = 0; b < nblocks; ++b) {
            const int32_t *k = &keys[5 * b];
            int64_t pk = pack_key(k[1], k[0], -k[2], -k[3], -k[4]);
            const int pb = kidx_new.find(pk);
            if (pb < 0) {
                set_error("gint_setup: internal error, partner block missing");
                return GINT_EINVAL;
            }
            partner[b] = pb;
            canon[b] = packed[b] <= pk;
        }
    }
    const KeyIndex &kidx = update_only ? old->kidx : kidx_new;
    const std::vector<int64_t> &offs = update_only ? old->offsets : offsets;
    const std::vector<uint8_t> &can = update_only ? old->canon : canon;
    const std::vector<int> &part = update_only ? old->partner : partner;

    // ---- batches and their atom-image slots, once per decomposition
    const BatchGeom bg = batch_geom(h);
    BatchSet sets[2];
    bool same[2] = {false, false};
    const int *dims[2] = {h->opt.batch, h->opt.batch_rho};
    for (int w = 0; w < 2; ++w) {
        // a position update writes into the storage the caller left in h->bs (earlier lists)
        if (update_only) take_storage(sets[w], h->bs[w]);
        for (int i = 0; i < 3; ++i) sets[w].dims[i] = dims[w][i];
        // vlocal batches of up to 64 points stay within 192 orbitals (two accumulators fit in
        // tensor memory); larger ones use the full 256 with one accumulator
        sets[w].limit_nb = (w == 0 && dims[w][0] * dims[w][1] * dims[w][2] <= 64) ? 192 : kMaxNb;
    }
    // the rho/force decomposition takes the padded density layout when every batch fits it (a
    // position update keeps the handle's layout and its split-store offsets)
    const bool padn1 = update_only ? old->bs[1].padn : true;
    ShareReq share;
    if (std::equal(dims[0], dims[0] + 3, dims[1]) && sets[0].limit_nb == sets[1].limit_nb) {
        share.soff = update_only ? &old->soff : &soff_pad;
        share.allow = !update_only || old->bs[1].shared;
        share.padn = padn1;
        share.old = update_only && old->bs[1].shared ? &old->bs[1] : nullptr;
        share.tbl2 = &sets[1].tbl2;
    }
    for (int w = 0; w < 2; ++w) {
        if (w == 1 && share.ok) {
            // the vlocal lists, tables and offsets; the slot-pair offsets are written already
            if (same[0]) {
                same[1] = true;
            } else {
                BatchSet &d = sets[1];
                const BatchSet &v = sets[0];
                par_copy(d.batches, v.batches);
                par_copy(d.slots, v.slots);
                par_copy(d.slot_img, v.slot_img);
                par_copy(d.tbl, v.tbl);
                par_copy(d.koff, v.koff);
                d.max_nb = v.max_nb;
                d.max_slots = v.max_slots;
                d.max_k = v.max_k;
                d.flops_dense = v.flops_dense;
            }
            sets[1].padn = padn1;
            sets[1].shared = true;
            continue;
        }
        bool padn = w == 1 && padn1, pad_fail = false;
        const std::vector<int> *soff = w == 0 ? nullptr : update_only ? &old->soff : padn ? &soff_pad : &soff_row;
        // a rho/force build of the vlocal batch shape starts from the vlocal batches
        const std::vector<BatchPart> *seed = w == 1 && share.soff && !share.parts.empty() ? &share.parts : nullptr;
        gint_status st = build_batches(h, tau, G, bg, rc, kidx, offs, can, part, soff, w == 0 ? &share : nullptr, seed,
                                       padn, &pad_fail, update_only ? &old->bs[w] : nullptr, &same[w], sets[w]);
        if (st != GINT_OK && pad_fail && update_only) {
            set_error("gint_update_positions: a batch no longer fits the padded density layout; build a new handle");
            return GINT_ESTATE;
        }
        if (st != GINT_OK && pad_fail) {
            padn = false;
            sets[w] = BatchSet{};
            for (int i = 0; i < 3; ++i) sets[w].dims[i] = dims[w][i];
            sets[w].limit_nb = kMaxNb;
            st = build_batches(h, tau, G, bg, rc, kidx, offs, can, part, &soff_row, nullptr, seed, false, nullptr,
                               nullptr, &same[w], sets[w]);
        }
        if (st != GINT_OK) return st;
        sets[w].padn = padn;
        sets[w].shared = false;
        if (!same[w] && sets[w].max_k + 32 > kMaxKCols) {
            set_error("gint_setup: a batch's padded orbital columns (%d) exceed %d", sets[w].max_k, kMaxKCols - 32);
            return GINT_EINVAL;
        }
    }
    if (update_only) {
        // a decomposition whose atom-image lists are unchanged gets new slot positions only, in
        // place (sets[w] holds the unused storage); one whose lists changed is replaced as a whole
        for (int w = 0; w < 2; ++w) {
            h->bs[w] = std::move(sets[w]);
            h->relist[w] = !same[w];
        }
    } else {
        h->keys = std::move(keys);
        h->offsets = std::move(offsets);
        h->partner = std::move(partner);
        h->canon = std::move(canon);
        h->kidx = std::move(kidx_new);
        const bool pad = sets[1].padn;
        h->soff = pad ? std::move(soff_pad) : std::move(soff_row);
        h->dms_plane = ((pad ? splane_pad : splane_row) + 7) / 8 * 8;
        for (int w = 0; w < 2; ++w) h->bs[w] = std::move(sets[w]);
    }
    h->tau.assign(tau, tau + 3 * natoms);
    h->plan.dV = std::fabs(G.det) / ((double)N1 * N2 * N3);
    for (int i = 0; i < 3; ++i)
        for (int c = 0; c < 3; ++c) h->plan.h[3 * i + c] = bg.h[3 * i + c];
    return GINT_OK;
}

// useful flops of the handle's vlocal decomposition: 2 n(r)^2 per point, n(r) = orbitals whose
// sphere contains r (exact count per point); per batch in parallel, summed in batch order
static double useful_flops(const gint_handle_s *h)
{
    const BatchSet &bs = h->bs[0];
    std::vector<double> fb(bs.batches.size(), 0.0);
    parallel_parts((int64_t)bs.batches.size(), host_threads(), [&](int64_t q0, int64_t q1, int) {
        for (int64_t q = q0; q < q1; ++q) {
            const Batch &B = bs.batches[q];
            int n1 = B.dims & 255, n2 = (B.dims >> 8) & 255, n3 = (B.dims >> 16) & 255;
            double f = 0.0;
            for (int a = 0; a < n1; ++a)
                for (int b = 0; b < n2; ++b)
                    for (int c = 0; c < n3; ++c) {
                        double off[3];
                        for (int x = 0; x < 3; ++x) off[x] = a * h->plan.h[x] + b * h->plan.h[3 + x] + c * h->plan.h[6 + x];
                        int n = 0;
                        for (int s = 0; s < B.nslots; ++s) {
                            const Slot &S = bs.slots[B.slot0 + s];
                            const double rc = h->plan.sp[S.species].rcut;
                            double d[3] = {S.d0[0] + off[0], S.d0[1] + off[1], S.d0[2] + off[2]};
                            double r2 = d[0] * d[0] + d[1] * d[1] + d[2] * d[2];
                            if (r2 < rc * rc) n += S.norb;
                        }
                        f += 2.0 * n * (double)n;
                    }
            fb[q] = f;
        }
    });
    double t = 0.0;
    for (double f : fb) t += f;
    return t;
}

// the handle's description (all but flops_useful, see useful_flops)
static void fill_info(gint_handle h)
{
    gint_info_t &info = h->info;
    const int64_t nblocks = (int64_t)h->keys.size() / 5;
    info.npts = (int64_t)h->grid[0] * h->grid[1] * h->grid[2];
    info.nblocks = nblocks;
    info.nvalues = h->offsets[nblocks];
    info.nbatches = (int64_t)h->bs[0].batches.size();
    info.nslots = (int64_t)h->bs[0].slots.size();
    info.max_orbitals = h->bs[0].max_nb;
    info.max_slots = h->bs[0].max_slots;
    info.dV = h->plan.dV;
    info.flops_dense = h->bs[0].flops_dense;
    info.nbatches_rho = (int64_t)h->bs[1].batches.size();
    info.max_orbitals_rho = h->bs[1].max_nb;
    info.nbasis = 0;
    for (int I = 0; I < h->natoms; ++I) info.nbasis += h->norb_atom[I];
    info.flops_dense_rho = h->bs[1].flops_dense;
    h->plan.nblocks = nblocks;
    h->plan.nvalues = info.nvalues;
}

// Estimated cost of one batch in a persistent tensor-core kernel.  The producers evaluate every
// orbital of the batch at every point (npts x nb), the epilogue handles the nb x nb result
// (vlocal: the upper triangle scattered into H) or the npts x nb result (rho: one dot product
// and, for the force, the orbital gradients per point); a fixed part covers barriers and the
// pipeline hand-offs.  The weights are relative clock-cycle costs measured per batch on Si and
// water workloads; only their ratios matter.
static double batch_cost(const Batch &B, int kind)
{
    const double np = (double)((B.dims & 255) * ((B.dims >> 8) & 255) * ((B.dims >> 16) & 255));
    const double nb = (double)B.nb;
    return kind == 0 ? 2000.0 + 2.6 * np * nb + 0.65 * nb * nb : 4000.0 + 4.0 * np * nb + 1.0 * nb * nb;
}

std::vector<int> partition_batches(const Batch *b, size_t n, int nparts, int kind)
{
    nparts = (int)std::min<size_t>((size_t)std::max(nparts, 1), std::max<size_t>(n, 1));
    std::vector<double> pre(n + 1, 0.0);
    for (size_t i = 0; i < n; ++i) pre[i + 1] = pre[i] + batch_cost(b[i], kind);
    std::vector<int> part(nparts + 1, 0);
    part[nparts] = (int)n;
    size_t j = 0;
    for (int k = 1; k < nparts; ++k) {
        const double target = pre[n] * k / nparts;
        while (j < n && pre[j + 1] <= target) ++j;
        // the boundary nearer to the target, keeping every range non-empty
        size_t cut = (j < n && target - pre[j] > pre[j + 1] - target) ? j + 1 : j;
        cut = std::max<size_t>(cut, (size_t)part[k - 1] + 1);
        cut = std::min<size_t>(cut, n - (size_t)(nparts - k));
        part[k] = (int)cut;
    }
    return part;
}

std::vector<int2> segment_ranges(const Batch *b, const std::vector<int> &seg, int npart, int kind)
{
    const int nseg = (int)seg.size() - 1;
    std::vector<int2> rng((size_t)nseg * npart, make_int2(0, 0));
    int rot = 0;
    for (int g = 0; g < nseg; ++g) {
        const int n = seg[g + 1] - seg[g];
        if (n == 0) continue;
        const std::vector<int> part = partition_batches(b + seg[g], (size_t)n, npart, kind);
        const int np = (int)part.size() - 1;
        for (int j = 0; j < np; ++j)
            rng[(size_t)g * npart + (j + rot) % npart] = make_int2(seg[g] + part[j], seg[g] + part[j + 1]);
        rot = (rot + np) % npart;
    }
    return rng;
}

}  // namespace gint

// ---------------------------------------------------------------------------------------
// gint_setup and the host-only entry points
// ---------------------------------------------------------------------------------------
using namespace gint;

template <class Vec>
static cudaError_t upload(void **dst, const Vec &v)
{
    using T = typename Vec::value_type;
    size_t bytes = std::max<size_t>(sizeof(T), v.size() * sizeof(T));
    cudaError_t e = cudaMalloc(dst, bytes);
    if (e != cudaSuccess) return e;
    if (!v.empty()) e = cudaMemcpy(*dst, v.data(), v.size() * sizeof(T), cudaMemcpyHostToDevice);
    return e;
}

// Copies v into the device array *dst of *cap bytes; an array v does not fit is replaced by one
// with an eighth of headroom, so that position updates (lists of about the same size) reuse it.
template <class Vec>
static cudaError_t upload_fit(void **dst, size_t *cap, const Vec &v)
{
    using T = typename Vec::value_type;
    const size_t bytes = v.size() * sizeof(T);
    if (!*dst || *cap < bytes) {
        if (*dst) cudaFree(*dst);
        *dst = nullptr;
        *cap = 0;
        const size_t want = std::max<size_t>(sizeof(T), bytes + bytes / 8);
        cudaError_t e = cudaMalloc(dst, want);
        if (e != cudaSuccess) return e;
        *cap = want;
    }
    return bytes ? cudaMemcpy(*dst, v.data(), bytes, cudaMemcpyHostToDevice) : cudaSuccess;
}

static void free_dev(gint_handle h)
{
    void *ptrs[] = {h->d_coef64, h->d_coef32, h->d_partner, h->d_blkoff, h->d_blkrows, h->d_status, h->d_dmsym,
                    h->d_dms, h->d_poff, h->d_red, h->d_hostio, h->bs[0].d_batches, h->bs[0].d_slots, h->bs[0].d_tbl,
                    h->bs[0].d_rng, h->bs[1].d_batches, h->bs[1].d_slots, h->bs[1].d_tbl, h->bs[1].d_rng,
                    h->bs[0].d_koff, h->bs[0].d_tbl2, h->bs[1].d_koff, h->bs[1].d_tbl2, h->bs[0].d_tslots,
                    h->bs[1].d_tslots, h->d_soff, h->d_env,
                    h->ks.d_keys, h->ks.d_grp, h->ks.d_pair, h->ks.d_colatom, h->ks.d_orboff, h->ks.d_kvec,
                    h->ks.d_phase, h->d_dm_scratch, h->d_dm_planes, h->d_amax};
    for (void *p : ptrs)
        if (p) cudaFree(p);
    for (cudaEvent_t &ev : h->io_ev)
        if (ev) cudaEventDestroy(ev);
    if (h->io_stream) cudaStreamDestroy(h->io_stream);
}

// the tensor-core kernels' records of a slot array (the FP64 kernels read the Slot records),
// written into the handle's staging array
static const hvec<TSlot> &tslots_of(gint_handle h, const hvec<Slot> &slots)
{
    hvec<TSlot> &t = h->tslot_stage;
    fit(t, slots.size());
    parallel_parts((int64_t)slots.size(), slots.size() < ((size_t)1 << 16) ? 1 : host_threads(),
                   [&](int64_t a, int64_t b, int) {
                       for (int64_t i = a; i < b; ++i) {
                           const Slot &S = slots[i];
                           TSlot &T = t[i];
                           T.atom = S.atom;
                           T.species = S.species;
                           T.orb_off = S.orb_off;
                           T.norb = S.norb;
                           for (int c = 0; c < 3; ++c) {
                               T.dh[c] = S.dh[c];
                               T.dl[c] = S.dl[c];
                           }
                       }
                   });
    return t;
}

// device arrays of one batch decomposition (replacing any earlier ones)
static gint_status upload_batchset(gint_handle h, int w)
{
    cudaError_t e;
    BatchSet &b = h->bs[w];
    // kernels still queued may read the arrays being replaced or overwritten
    if (b.d_batches && (e = cudaDeviceSynchronize()) != cudaSuccess) return cuda_fail(e, "synchronise");
    size_t *c = b.d_cap;
    if ((e = upload_fit(&b.d_batches, &c[0], b.batches)) != cudaSuccess) return cuda_fail(e, "upload batches");
    if ((e = upload_fit(&b.d_slots, &c[1], b.slots)) != cudaSuccess) return cuda_fail(e, "upload slots");
    if ((e = upload_fit(&b.d_tbl, &c[2], b.tbl)) != cudaSuccess) return cuda_fail(e, "upload tables");
    if ((e = upload_fit(&b.d_koff, &c[4], b.koff)) != cudaSuccess) return cuda_fail(e, "upload K offsets");
    if ((e = upload_fit(&b.d_tbl2, &c[5], b.tbl2)) != cudaSuccess) return cuda_fail(e, "upload split tables");
    if ((e = upload_fit(&b.d_tslots, &c[6], tslots_of(h, b.slots))) != cudaSuccess) return cuda_fail(e, "upload slots");
    const int nb = (int)b.batches.size();
    b.rng = segment_ranges(b.batches.data(), {0, nb}, std::max(1, std::min(h->nsm, nb)), w);
    if ((e = upload_fit(&b.d_rng, &c[3], b.rng)) != cudaSuccess) return cuda_fail(e, "upload CTA ranges");
    return GINT_OK;
}

static gint_status upload_geometry(gint_handle h)
{
    cudaError_t e;
    gint_status st;
    // (re)upload everything that depends on positions; the block layout is fixed after set-up
    if (!h->d_blkoff) {
        for (int w = 0; w < 2; ++w)
            if ((st = upload_batchset(h, w)) != GINT_OK) return st;
        if ((e = upload(&h->d_partner, h->partner)) != cudaSuccess) return cuda_fail(e, "upload partner");
        if ((e = upload(&h->d_soff, h->soff)) != cudaSuccess) return cuda_fail(e, "upload split offsets");
        if ((e = upload(&h->d_blkoff, h->offsets)) != cudaSuccess) return cuda_fail(e, "upload offsets");
        std::vector<int> rows(h->info.nblocks);
        for (int64_t b = 0; b < h->info.nblocks; ++b) rows[b] = h->norb_atom[h->keys[5 * b]];
        if ((e = upload(&h->d_blkrows, rows)) != cudaSuccess) return cuda_fail(e, "upload rows");
    } else {
        for (int w = 0; w < 2; ++w) {
            BatchSet &b = h->bs[w];
            if (h->relist[w]) {
                if ((st = upload_batchset(h, w)) != GINT_OK) return st;
                h->relist[w] = false;
                continue;
            }
            if (b.slots.empty()) continue;
            e = cudaMemcpy(b.d_slots, b.slots.data(), b.slots.size() * sizeof(Slot), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "update slots");
            const hvec<TSlot> &ts = tslots_of(h, b.slots);
            e = cudaMemcpy(b.d_tslots, ts.data(), ts.size() * sizeof(TSlot), cudaMemcpyHostToDevice);
            if (e != cudaSuccess) return cuda_fail(e, "update slots");
        }
    }
    Plan &P = h->plan;
    P.partner = (const int *)h->d_partner;
    P.blk_off = (const int64_t *)h->d_blkoff;
    P.blk_rows = (const int *)h->d_blkrows;
    return GINT_OK;
}

extern "C" gint_status gint_setup(gint_handle *out, const double cell[9], int natoms, const int *species,
                                  const double *tau, int nspecies, const gint_species *sp, const int grid[3],
                                  const gint_options *opt)
{
    if (!out || !cell || !species || !tau || !sp || !grid) {
        set_error("gint_setup: null argument");
        return GINT_EINVAL;
    }
    *out = nullptr;
    if (natoms < 1 || natoms >= (1 << 20) || nspecies < 1 || nspecies > kMaxSpecies) {
        set_error("gint_setup: natoms must be in [1, 2^20) and nspecies in [1, %d]", kMaxSpecies);
        return GINT_EINVAL;
    }
    for (int i = 0; i < 3; ++i)
        if (grid[i] < 1 || grid[i] > (1 << 14)) {
            set_error("gint_setup: grid dimension %d out of range", grid[i]);
            return GINT_EINVAL;
        }
    for (int i = 0; i < 9; ++i)
        if (!std::isfinite(cell[i])) {
            set_error("gint_setup: non-finite cell");
            return GINT_EINVAL;
        }
    Geo G = make_geo(cell);
    if (!(std::fabs(G.det) > 1e-8)) {
        set_error("gint_setup: singular cell");
        return GINT_EINVAL;
    }
    for (int i = 0; i < natoms; ++i) {
        if (species[i] < 0 || species[i] >= nspecies) {
            set_error("gint_setup: species[%d] = %d out of range", i, species[i]);
            return GINT_EINVAL;
        }
        for (int c = 0; c < 3; ++c)
            if (!std::isfinite(tau[3 * i + c])) {
                set_error("gint_setup: non-finite position of atom %d", i);
                return GINT_EINVAL;
            }
    }
    gint_options o{};
    o.batch[0] = 4; o.batch[1] = 4; o.batch[2] = 4;
    o.batch_rho[0] = 4; o.batch_rho[1] = 4; o.batch_rho[2] = 8;
    if (opt) {
        for (int i = 0; i < 3; ++i) {
            if (opt->batch[i] > 0) o.batch[i] = opt->batch[i];
            if (opt->batch_rho[i] > 0) o.batch_rho[i] = opt->batch_rho[i];
        }
        if (opt->wait_budget < 0) {
            set_error("gint_setup: negative wait_budget");
            return GINT_EINVAL;
        }
        o.wait_budget = opt->wait_budget;
    }
    for (const int *b : {o.batch, o.batch_rho})
        if (b[0] > kMaxBatchDim || b[1] > kMaxBatchDim || b[2] > kMaxBatchDim || b[0] * b[1] * b[2] > kMaxBatchPts ||
            (b[2] % 2)) {
            set_error("gint_setup: batch %dx%dx%d invalid (<= %d per axis, <= %d points, even along a3)", b[0], b[1],
                      b[2], kMaxBatchDim, kMaxBatchPts);
            return GINT_EINVAL;
        }
    // device
    int dev = 0;
    cudaError_t e = cudaGetDevice(&dev);
    if (e != cudaSuccess) return cuda_fail(e, "gint_setup: no CUDA device");
    cudaDeviceProp prop;
    if ((e = cudaGetDeviceProperties(&prop, dev)) != cudaSuccess) return cuda_fail(e, "gint_setup");
    if (prop.major * 10 + prop.minor != 103) {
        set_error("gint_setup: device %d is sm_%d%d; this library is built for sm_103a only", dev, prop.major,
                  prop.minor);
        return GINT_ECUDA;
    }

    gint_handle h = new gint_handle_s();
    h->device = dev;
    h->nsm = prop.multiProcessorCount;
    memcpy(h->cell, cell, sizeof(h->cell));
    for (int i = 0; i < 3; ++i) h->grid[i] = grid[i];
    h->natoms = natoms;
    h->nspecies = nspecies;
    h->species.assign(species, species + natoms);
    h->opt = o;
    Plan &P = h->plan;
    P.natoms = natoms;
    P.nspecies = nspecies;
    for (int i = 0; i < 3; ++i) P.grid[i] = grid[i];
    P.npts = (int64_t)grid[0] * grid[1] * grid[2];
    P.spin_limit = o.wait_budget > 0 ? (long long)o.wait_budget : 4000000000LL;   // default about 2 s at 2 GHz

    // species and splines
    std::vector<double> coef64;
    std::vector<float4> coef32;
    for (int s = 0; s < nspecies; ++s) {
        const gint_species &S = sp[s];
        if (S.nrad < 1 || S.nrad > kMaxRad || !S.l || !S.ftab || !S.dfdr0 || !(S.rcut > 0) || !(S.dr > 0) ||
            S.ntab < 3) {
            set_error("gint_setup: species %d invalid (nrad 1..%d, tables, rcut > 0, dr > 0, ntab >= 3)", s, kMaxRad);
            delete h;
            return GINT_EINVAL;
        }
        if ((S.ntab - 1) * S.dr < S.rcut * (1.0 - 1e-12)) {
            set_error("gint_setup: species %d table ends at %g < rcut %g", s, (S.ntab - 1) * S.dr, S.rcut);
            delete h;
            return GINT_EINVAL;
        }
        DevSpecies &D = P.sp[s];
        D.nrad = S.nrad;
        D.nint = S.ntab - 1;
        D.coef_off = (int)(coef64.size() / 4);
        D.rcut = S.rcut;
        D.inv_dr = 1.0 / S.dr;
        D.rcut_f = (float)S.rcut;
        D.inv_dr_f = (float)(1.0 / S.dr);
        int norb = 0;
        for (int r = 0; r < S.nrad; ++r) {
            if (S.l[r] < 0 || S.l[r] > 2) {
                set_error("gint_setup: species %d radial %d has l = %d (supported: 0..2)", s, r, S.l[r]);
                delete h;
                return GINT_EINVAL;
            }
            D.l[r] = S.l[r];
            norb += 2 * S.l[r] + 1;
        }
        if (norb > kMaxOrbSpecies) {
            set_error("gint_setup: species %d has %d orbitals (max %d)", s, norb, kMaxOrbSpecies);
            delete h;
            return GINT_EINVAL;
        }
        D.norb = norb;
        for (int i = 0; i < S.nrad * S.ntab; ++i)
            if (!std::isfinite(S.ftab[i])) {
                set_error("gint_setup: species %d table has a non-finite value", s);
                delete h;
                return GINT_EINVAL;
            }
        // slopes per radial, then interval-major records
        std::vector<std::vector<double>> k(S.nrad);
        for (int r = 0; r < S.nrad; ++r) spline_slopes(S.ftab + (size_t)r * S.ntab, S.ntab, S.dr, S.dfdr0[r], 0.0, k[r]);
        for (int i = 0; i < S.ntab - 1; ++i)
            for (int r = 0; r < S.nrad; ++r) {
                const double *y = S.ftab + (size_t)r * S.ntab;
                double hh = S.dr;
                double c0 = y[i], c1 = hh * k[r][i];
                double c2 = 3.0 * (y[i + 1] - y[i]) - hh * (2.0 * k[r][i] + k[r][i + 1]);
                double c3 = 2.0 * (y[i] - y[i + 1]) + hh * (k[r][i] + k[r][i + 1]);
                coef64.insert(coef64.end(), {c0, c1, c2, c3});
                coef32.push_back(make_float4((float)c0, (float)c1, (float)c2, (float)c3));
            }
    }
    h->norb_atom.resize(natoms);
    for (int i = 0; i < natoms; ++i) h->norb_atom[i] = P.sp[species[i]].norb;

    gint_status st = build_geometry(h, tau, nullptr);
    if (st != GINT_OK) {
        delete h;
        return st;
    }
    fill_info(h);
    h->info.flops_useful = useful_flops(h);
    if ((e = upload(&h->d_coef64, coef64)) != cudaSuccess || (e = upload(&h->d_coef32, coef32)) != cudaSuccess) {
        free_dev(h);
        delete h;
        return cuda_fail(e, "gint_setup: upload splines");
    }
    P.coef64 = (const double *)h->d_coef64;
    P.coef32 = (const float4 *)h->d_coef32;
    h->coef32_host = coef32;
    {
        // |phi| <= max |f| * max |Y_lm|; on an interval |f(t)| <= |c0| + |c1| + |c2| + |c3|
        // (0 <= t <= 1), and |Y_lm| <= sqrt(5/(16 pi)) * 2 = 0.631 for l <= 2
        double fmax = 0.0;
        for (size_t i = 0; i + 3 < coef64.size(); i += 4)
            fmax = std::max(fmax, std::fabs(coef64[i]) + std::fabs(coef64[i + 1]) + std::fabs(coef64[i + 2]) +
                                      std::fabs(coef64[i + 3]));
        h->phimax = (float)(fmax * 0.64);
        // per species and interval i: max over intervals j >= i and radials of the interval
        // bound, times the Y_lm bound (non-increasing in r)
        for (int s = 0; s < nspecies; ++s) {
            DevSpecies &D = P.sp[s];
            D.env_off = (int)h->env_host.size();
            std::vector<float> env(D.nint);
            double run = 0.0;
            for (int i = D.nint - 1; i >= 0; --i) {
                for (int r = 0; r < D.nrad; ++r) {
                    const double *c = &coef64[4 * ((size_t)D.coef_off + (size_t)i * D.nrad + r)];
                    run = std::max(run, std::fabs(c[0]) + std::fabs(c[1]) + std::fabs(c[2]) + std::fabs(c[3]));
                }
                env[i] = (float)(run * 0.64 * 1.0001);
            }
            h->env_host.insert(h->env_host.end(), env.begin(), env.end());
        }
    }
    if ((e = upload(&h->d_env, h->env_host)) != cudaSuccess) {
        free_dev(h);
        delete h;
        return cuda_fail(e, "gint_setup: upload envelopes");
    }
    P.env = (const float *)h->d_env;
    if ((st = upload_geometry(h)) != GINT_OK) {
        free_dev(h);
        delete h;
        return st;
    }
    if ((e = cudaMalloc((void **)&h->d_status, sizeof(int))) != cudaSuccess ||
        (e = cudaMemset(h->d_status, 0, sizeof(int))) != cudaSuccess ||
        (e = cudaMalloc((void **)&h->d_dmsym, std::max<size_t>(8, h->info.nvalues * sizeof(double)))) != cudaSuccess ||
        (e = cudaMalloc((void **)&h->d_dms, std::max<size_t>(16, (size_t)h->dms_plane * 8))) != cudaSuccess ||
        (e = cudaMalloc((void **)&h->d_red, 4096 * sizeof(double))) != cudaSuccess ||
        (e = cudaMalloc((void **)&h->d_amax, 4 * sizeof(float))) != cudaSuccess ||
        (e = cudaMemset(h->d_amax, 0, 4 * sizeof(float))) != cudaSuccess) {
        free_dev(h);
        delete h;
        return cuda_fail(e, "gint_setup: allocate");
    }
    {
        // offsets a h1 + b h2 + c h3 of local grid points, FP64 then split into FP32 hi + lo
        std::vector<float> tab((size_t)kPoffDim * kPoffDim * kPoffDim * 6);
        for (int a = 0; a < kPoffDim; ++a)
            for (int b = 0; b < kPoffDim; ++b)
                for (int c = 0; c < kPoffDim; ++c) {
                    float *t = &tab[(((size_t)a * kPoffDim + b) * kPoffDim + c) * 6];
                    for (int q = 0; q < 3; ++q) {
                        double v = a * P.h[q] + b * P.h[3 + q] + c * P.h[6 + q];
                        t[q] = (float)v;
                        t[3 + q] = (float)(v - (double)t[q]);
                    }
                }
        if ((e = upload((void **)&h->d_poff, tab)) != cudaSuccess) {
            free_dev(h);
            delete h;
            return cuda_fail(e, "gint_setup: point offsets");
        }
        P.poff = h->d_poff;
    }
    P.status = h->d_status;
    *out = h;
    return GINT_OK;
}

extern "C" gint_status gint_destroy(gint_handle h)
{
    if (!h) return GINT_OK;
    free_dev(h);
    delete h;
    return GINT_OK;
}

extern "C" gint_status gint_block_layout(gint_handle h, int64_t *nblocks, int64_t *nvalues, const int32_t **keys,
                                         const int64_t **offsets)
{
    if (!h) {
        set_error("gint_block_layout: null handle");
        return GINT_EINVAL;
    }
    if (nblocks) *nblocks = h->info.nblocks;
    if (nvalues) *nvalues = h->info.nvalues;
    if (keys) *keys = h->keys.data();
    if (offsets) *offsets = h->offsets.data();
    return GINT_OK;
}

extern "C" gint_status gint_get_info(gint_handle h, gint_info_t *info)
{
    if (!h || !info) {
        set_error("gint_get_info: null argument");
        return GINT_EINVAL;
    }
    if (h->flops_stale) {
        h->info.flops_useful = useful_flops(h);
        h->flops_stale = false;
    }
    *info = h->info;
    return GINT_OK;
}

extern "C" gint_status gint_update_positions(gint_handle h, const double *tau)
{
    if (!h || !tau) {
        set_error("gint_update_positions: null argument");
        return GINT_EINVAL;
    }
    for (int i = 0; i < 3 * h->natoms; ++i)
        if (!std::isfinite(tau[i])) {
            set_error("gint_update_positions: non-finite position");
            return GINT_EINVAL;
        }
    // build into a scratch handle (compared with this one) so a topology change leaves the
    // handle untouched; the lists are written into the storage the previous update replaced
    gint_handle_s tmp;
    tmp.plan = h->plan;
    memcpy(tmp.cell, h->cell, sizeof(tmp.cell));
    memcpy(tmp.grid, h->grid, sizeof(tmp.grid));
    tmp.natoms = h->natoms;
    tmp.nspecies = h->nspecies;
    tmp.species = h->species;
    tmp.norb_atom = h->norb_atom;
    tmp.opt = h->opt;
    for (int w = 0; w < 2; ++w) {
        take_storage(tmp.bs[w], h->spare[w]);
        tmp.bs[w].limit_nb = h->bs[w].limit_nb;
    }
    gint_status st = build_geometry(&tmp, tau, h);
    if (st != GINT_OK) {
        for (int w = 0; w < 2; ++w) take_storage(h->spare[w], tmp.bs[w]);
        return st;
    }
    cudaError_t e = cudaSetDevice(h->device);
    if (e != cudaSuccess) return cuda_fail(e, "gint_update_positions");
    for (int w = 0; w < 2; ++w) {
        h->relist[w] = tmp.relist[w];
        BatchSet &o = h->bs[w];
        if (tmp.relist[w]) {
            // the new lists, with the old device arrays (refilled, or replaced where too small, by
            // upload_geometry);
            // the old host arrays become the storage of the next update
            void *dev[7] = {o.d_batches, o.d_slots, o.d_tbl, o.d_rng, o.d_koff, o.d_tbl2, o.d_tslots};
            size_t cap[7];
            memcpy(cap, o.d_cap, sizeof(cap));
            take_storage(h->spare[w], o);
            o = std::move(tmp.bs[w]);
            memcpy(o.d_cap, cap, sizeof(cap));
            o.d_batches = dev[0];
            o.d_slots = dev[1];
            o.d_tbl = dev[2];
            o.d_rng = dev[3];
            o.d_koff = dev[4];
            o.d_tbl2 = dev[5];
            o.d_tslots = dev[6];
        } else {
            take_storage(h->spare[w], tmp.bs[w]);
            place_slots(h, o, tau);
        }
    }
    h->tau = std::move(tmp.tau);
    h->plan.dV = tmp.plan.dV;
    fill_info(h);
    h->flops_stale = true;   // recounted when the description is next read
    return upload_geometry(h);
}

extern "C" const char *gint_last_error(void) { return gint::last_error(); }
