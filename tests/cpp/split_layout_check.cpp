// Host-side checks of the tiler (make_tiling: partitions, caps, CTA ranges),
// of the split interface layout (make_split_form) and of the tiler's warp
// alignment for it, without a GPU.  Builds random local
// matrices over overlapping node sets, lays them out for several warp row
// counts and verifies every invariant the sweep kernel relies on.  Prints
// "ok" and returns 0, or prints the first violation and returns 1.
#include <cmath>
#include <cstdio>
#include <cstdint>
#include <vector>

#include "jac_internal.h"

using namespace jac;

static uint64_t rng_state = 0x9e3779b97f4a7c15ull;
static uint64_t next_u64()
{
    rng_state += 0x9e3779b97f4a7c15ull;
    uint64_t z = rng_state;
    z = (z ^ (z >> 30)) * 0xbf58476d1ce4e5b9ull;
    z = (z ^ (z >> 27)) * 0x94d049bb133111ebull;
    return z ^ (z >> 31);
}
static double uniform() { return (double)(next_u64() >> 11) * (1.0 / 9007199254740992.0); }

#define CHECK(cond, ...)                          \
    do {                                          \
        if (!(cond)) {                            \
            std::printf("FAIL: " __VA_ARGS__);    \
            std::printf("\n");                    \
            return 1;                             \
        }                                         \
    } while (0)

struct Local {
    std::vector<int32_t> rowptr, col, l2g;
    std::vector<double> val;
};

static int check_case(int64_t n, int nsub, int max_extra, int warp_rows)
{
    // node sets: every node to one owner, some to up to max_extra more subdomains
    std::vector<std::vector<int32_t>> sets(nsub);
    std::vector<int> mult(n, 0);
    for (int64_t g = 0; g < n; ++g) {
        const int s0 = (int)(next_u64() % nsub);
        sets[s0].push_back((int32_t)g);
        mult[g] = 1;
        if (uniform() < 0.3) {
            const int extra = 1 + (int)(next_u64() % max_extra);
            for (int e = 0; e < extra; ++e) {
                const int s = (int)(next_u64() % nsub);
                bool have = false;
                for (int32_t v : sets[s]) have |= (v == g);
                if (!have) { sets[s].push_back((int32_t)g); ++mult[g]; }
            }
        }
    }
    std::vector<Local> L(nsub);
    std::vector<jac_local> sub(nsub);
    for (int s = 0; s < nsub; ++s) {
        Local& l = L[s];
        const int nl = (int)sets[s].size();
        l.l2g = sets[s];
        l.rowptr.push_back(0);
        for (int r = 0; r < nl; ++r) {
            for (int k = 0; k < 5 && nl > 1; ++k) {
                int c = (int)(next_u64() % nl);
                if (c == r) continue;
                l.col.push_back(c);
                l.val.push_back(uniform() - 0.5);
            }
            l.col.push_back(r);
            l.val.push_back(4.0 + uniform());
            l.rowptr.push_back((int32_t)l.col.size());
        }
        sub[s] = jac_local{nl, (int64_t)l.col.size(), l.rowptr.data(), l.col.data(), l.val.data(), l.l2g.data()};
    }
    int maxm = 0;
    for (int64_t g = 0; g < n; ++g) maxm = mult[g] > maxm ? mult[g] : maxm;
    SplitForm f;
    Error e = make_split_form(n, nsub, sub.data(), warp_rows, f);
    if (maxm > warp_rows) {
        CHECK(!e.ok() && e.st == JAC_EINVAL, "a row in %d subdomains must be rejected at %d warp rows", maxm, warp_rows);
        return 0;
    }
    CHECK(e.ok(), "make_split_form: %s", e.msg.c_str());
    const ScaledForm& tf = f.tf;
    // new order: interiors by subdomain, then the interface, ascending within each
    int64_t n_ifc = 0;
    for (int64_t g = 0; g < n; ++g) n_ifc += mult[g] >= 2;
    CHECK(f.n_ifc == n_ifc && f.n_own == n - n_ifc, "interface count %lld vs %lld", (long long)f.n_ifc,
          (long long)n_ifc);
    for (int64_t r = 0; r < n; ++r) CHECK(f.plan.iperm[f.plan.perm[r]] == r, "perm/iperm mismatch at %lld", (long long)r);
    for (int64_t r = f.n_own + 1; r < n; ++r) CHECK(f.plan.perm[r] > f.plan.perm[r - 1], "interface not ascending");
    // assembled diagonal
    std::vector<double> d(n, 0.0);
    for (int s = 0; s < nsub; ++s)
        for (int r = 0; r < sub[s].n; ++r)
            for (int k = L[s].rowptr[r]; k < L[s].rowptr[r + 1]; ++k)
                if (L[s].col[k] == r) d[L[s].l2g[r]] += L[s].val[k];
    for (int64_t r = 0; r < n; ++r) CHECK(tf.d[r] == d[f.plan.perm[r]], "assembled diagonal of new row %lld", (long long)r);
    // slot rows: groups consecutive, in subdomain order, never across a warp
    CHECK((int64_t)f.slot_info.size() == tf.n - f.n_own, "slot_info size");
    CHECK((int64_t)f.bmap.size() == tf.n, "bmap size");
    for (int64_t r = 0; r < f.n_own; ++r) CHECK(f.bmap[r] == f.plan.perm[r], "bmap of interior row");
    int64_t seen = 0, partials = 0;
    for (int64_t p = 0; p < tf.n - f.n_own;) {
        const uint32_t info = f.slot_info[p];
        if (info == 0) {   // padding row: empty, no b
            CHECK(tf.rowptr[f.n_own + p + 1] == tf.rowptr[f.n_own + p], "padding row not empty");
            CHECK(f.bmap[f.n_own + p] == -1, "padding row has b");
            ++p;
            continue;
        }
        const int m = (int)(info & 63u);
        const int64_t i = (int64_t)(info >> 6);
        CHECK(i == seen, "interface rows out of order (%lld, expected %lld)", (long long)i, (long long)seen);
        const int64_t g = f.plan.perm[f.n_own + i];
        CHECK(m == mult[g], "group size %d vs multiplicity %d", m, mult[g]);
        CHECK(p % warp_rows + m <= warp_rows, "group of row %lld straddles a warp", (long long)g);
        CHECK(f.bmap[f.n_own + p] == g, "leader's b");
        for (int q = 1; q < m; ++q) {
            CHECK(f.slot_info[p + q] == 0u, "non-leader slot carries a descriptor");
            CHECK(f.bmap[f.n_own + p + q] == -1, "non-leader slot has b");
        }
        partials += m;
        ++seen;
        p += m;
    }
    CHECK(seen == n_ifc && partials == f.partials, "groups %lld of %lld", (long long)seen, (long long)n_ifc);
    // entries: columns in range, S = -a / d_col
    for (int64_t e2 = 0; e2 < (int64_t)tf.col.size(); ++e2) {
        CHECK(tf.col[e2] >= 0 && tf.col[e2] < n, "column out of range");
        CHECK(std::isfinite(tf.S[e2]), "S not finite");
    }
    // tiling: cuts at and after n_own fall on warp boundaries, none crosses n_own
    for (int64_t ctas : {7, 64, 301}) {
        Tiling t;
        make_tiling(tf, f.plan, 256, 1536, ctas, t, nullptr, f.n_own, warp_rows);
        for (int64_t i2 = 0; i2 < t.ntiles(); ++i2) {
            const int64_t r0 = t.row0[i2], r1 = t.row0[i2 + 1];
            CHECK(r1 > r0, "empty tile");
            CHECK(!(r0 < f.n_own && r1 > f.n_own), "tile crosses the interior/slot boundary");
            if (r0 >= f.n_own) CHECK((r0 - f.n_own) % warp_rows == 0, "slot tile starts off a warp boundary");
        }
        CHECK(t.row0.back() == tf.n, "tiles do not cover the kernel rows");
    }
    // split tiling: interior tiles then slot tiles, each CTA a range of both
    for (int64_t ctas : {1, 7, 64, 301}) {
        Tiling t;
        make_split_tiling(f, 256, 1536, ctas, t);
        const int64_t T = t.ntiles();
        CHECK(t.row0.front() == 0 && t.row0.back() == tf.n, "split tiles do not cover the kernel rows");
        CHECK((int64_t)t.cta0.size() == ctas + 1 && (int64_t)t.cta1.size() == ctas + 1, "CTA range arrays");
        const int64_t T1 = t.cta0[ctas];
        CHECK(t.cta0[0] == 0 && t.cta1[0] == T1 && t.cta1[ctas] == T, "CTA ranges do not cover the tiles");
        for (int64_t g = 0; g < ctas; ++g)
            CHECK(t.cta0[g + 1] >= t.cta0[g] && t.cta1[g + 1] >= t.cta1[g], "CTA ranges not monotone");
        CHECK(T1 == 0 || t.row0[T1] == f.n_own, "interior tiles end at %lld, not at n_own", (long long)t.row0[T1]);
        for (int64_t i2 = 0; i2 < T; ++i2) {
            const int64_t r0 = t.row0[i2], r1 = t.row0[i2 + 1];
            CHECK(r1 > r0, "empty split tile");
            CHECK(t.nnz0[i2] == tf.rowptr[r0], "split tile entry offset");
            if (i2 < T1) CHECK(r1 <= f.n_own, "an interior-range tile holds slot rows");
            else CHECK(r0 >= f.n_own && (r0 - f.n_own) % warp_rows == 0, "slot tile off a warp boundary");
        }
    }
    return 0;
}

// General tiling (make_plan / make_scaled_form / make_tiling on a CSR with
// irregular rows, some longer than a tile's entry cap).
static int check_tiling(int64_t n, jac_splitting sp, int32_t nparts, int32_t rows_per_tile, int32_t max_entries,
                        int64_t ctas)
{
    HostCSR M;
    M.n = n;
    M.rowptr.assign(1, 0);
    for (int64_t r = 0; r < n; ++r) {
        int64_t len = 1 + (int64_t)(next_u64() % 12);
        if (next_u64() % 500 == 0) len = 2 * max_entries + (int64_t)(next_u64() % 100);   // oversized
        for (int64_t k = 0; k < len && k < n - 1; ++k) {
            int64_t c = (int64_t)(next_u64() % n);
            if (c == r) c = (c + 1) % n;
            M.col.push_back((int32_t)c);
            M.val.push_back(-0.01);
        }
        M.col.push_back((int32_t)r);
        M.val.push_back(100.0);
        M.rowptr.push_back((int32_t)M.col.size());
    }
    jac_opts o{};   // band splittings read no option (node_of_row NULL: row r at node r)
    Plan plan;
    Error e = make_plan(M, sp, nparts, o, plan);
    CHECK(e.ok(), "make_plan: %s", e.msg.c_str());
    ScaledForm tf;
    e = make_scaled_form(M, plan, tf);
    CHECK(e.ok(), "make_scaled_form: %s", e.msg.c_str());
    Tiling t;
    make_tiling(tf, plan, rows_per_tile, max_entries, ctas, t, nullptr);
    CHECK((int64_t)t.cta0.size() == ctas + 1 && t.cta0[0] == 0 && t.cta0[ctas] == t.ntiles(), "CTA ranges");
    for (int64_t g = 0; g < ctas; ++g) CHECK(t.cta0[g + 1] >= t.cta0[g], "CTA ranges not monotone");
    CHECK(t.row0.front() == 0 && t.row0.back() == n, "tiles do not cover the rows");
    size_t p = 0;
    for (int64_t i = 0; i < t.ntiles(); ++i) {
        const int64_t r0 = t.row0[i], r1 = t.row0[i + 1];
        CHECK(r1 > r0 && r1 - r0 <= rows_per_tile, "tile rows %lld", (long long)(r1 - r0));
        while (p + 1 < plan.part_ptr.size() && plan.part_ptr[p + 1] <= r0) ++p;
        CHECK(r1 <= plan.part_ptr[p + 1], "tile crosses a partition");
        const int64_t ent = tf.rowptr[r1] - tf.rowptr[r0];
        CHECK(ent <= max_entries || r1 - r0 == 1, "tile of %lld rows holds %lld entries", (long long)(r1 - r0),
              (long long)ent);
        CHECK(t.nnz0[i] == tf.rowptr[r0], "entry offset");
    }
    return 0;
}

int main()
{
    for (int trial = 0; trial < 8; ++trial) {
        const int64_t n = 1000 + (int64_t)(next_u64() % 20000);
        const jac_splitting sp = trial % 2 ? JAC_BANDROW_NNZ : JAC_BANDROW;
        const int32_t nparts = 1 + (int32_t)(next_u64() % 64);
        const int32_t rows = trial % 3 == 0 ? 128 : 256;
        const int32_t cap = 300 + (int32_t)(next_u64() % 2000);
        const int64_t ctas = 1 + (int64_t)(next_u64() % 456);
        if (check_tiling(n, sp, nparts, rows, cap, ctas)) {
            std::printf("  (tiling trial %d, n %lld, parts %d, rows %d, cap %d, ctas %lld)\n", trial, (long long)n,
                        nparts, rows, cap, (long long)ctas);
            return 1;
        }
    }
    const int warp_rows[] = {32, 16, 8};
    for (int trial = 0; trial < 12; ++trial)
        for (int w : warp_rows) {
            const int64_t n = 200 + (int64_t)(next_u64() % 3000);
            const int nsub = 2 + (int)(next_u64() % 40);
            const int max_extra = 1 + (int)(next_u64() % 12);
            if (check_case(n, nsub, max_extra, w)) {
                std::printf("  (trial %d, n %lld, nsub %d, warp rows %d)\n", trial, (long long)n, nsub, w);
                return 1;
            }
        }
    std::printf("ok\n");
    return 0;
}
