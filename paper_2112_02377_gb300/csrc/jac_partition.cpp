// Host-side splitting, reordering, dependency lists and tiling.
//
// Paper: band-row splitting (Sec. 4.2), the sparsity-pattern splitting with
// receive/send dependency lists and nnz-weighted balancing (Sec. 4.2.2), and
// substructuring with subdomain interiors first and the interface block last
// (Sec. 4.3, block form Eq. (4.4)).
#include <algorithm>
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <numeric>

#include "jac_internal.h"

namespace jac {

static std::string fmt(const char* f, long long a = 0, long long b = 0, long long c = 0)
{
    char buf[256];
    std::snprintf(buf, sizeof(buf), f, a, b, c);
    return buf;
}

Error host_csr_from_abi(const jac_csr* A, bool transpose, HostCSR& out)
{
    if (!A) return Error(JAC_EINVAL, "A is NULL");
    if (A->n < 1) return Error(JAC_EINVAL, "n must be >= 1 (empty system)");
    if (A->n >= (int64_t)INT32_MAX) return Error(JAC_EINVAL, "n must be < 2^31-1");
    if (A->nnz < 0 || A->nnz >= (int64_t)INT32_MAX) return Error(JAC_EINVAL, "nnz must be in [0, 2^31-1)");
    if (A->index_base != 0 && A->index_base != 1) return Error(JAC_EINVAL, "index_base must be 0 or 1");
    if (A->nnz > 0 && (!A->col || !A->val)) return Error(JAC_EINVAL, "col/val are NULL");
    if (!A->rowptr) return Error(JAC_EINVAL, "rowptr is NULL");
    const int64_t n = A->n, base = A->index_base;
    if (A->rowptr[0] != base) return Error(JAC_EINVAL, "rowptr[0] must equal index_base");
    if ((int64_t)A->rowptr[n] - base != A->nnz) return Error(JAC_EINVAL, "rowptr[n] - index_base must equal nnz");
    HostCSR M;
    M.n = n;
    M.rowptr.resize(n + 1);
    for (int64_t i = 0; i <= n; ++i) {
        int64_t v = (int64_t)A->rowptr[i] - base;
        if (i > 0 && v < M.rowptr[i - 1]) return Error(JAC_EINVAL, fmt("rowptr decreases at row %lld", i));
        M.rowptr[i] = (int32_t)v;
    }
    M.col.resize(A->nnz);
    M.val.resize(A->nnz);
    for (int64_t k = 0; k < A->nnz; ++k) {
        int64_t c = (int64_t)A->col[k] - base;
        if (c < 0 || c >= n) return Error(JAC_EINVAL, fmt("column index out of range at entry %lld", k));
        if (!std::isfinite(A->val[k])) return Error(JAC_EINVAL, fmt("non-finite value at entry %lld", k));
        M.col[k] = (int32_t)c;
        M.val[k] = A->val[k];
    }
    out = transpose ? transpose_csr(M) : std::move(M);
    return Error();
}

HostCSR transpose_csr(const HostCSR& A)
{
    // Counting sort by column; rows of A^T list their entries in ascending
    // original row order (stable for repeated (i, j) pairs).
    HostCSR T;
    T.n = A.n;
    const int64_t nnz = A.nnz();
    T.rowptr.assign(A.n + 1, 0);
    for (int64_t k = 0; k < nnz; ++k) T.rowptr[A.col[k] + 1]++;
    for (int64_t i = 0; i < A.n; ++i) T.rowptr[i + 1] += T.rowptr[i];
    std::vector<int32_t> fill(T.rowptr.begin(), T.rowptr.end() - 1);
    T.col.resize(nnz);
    T.val.resize(nnz);
    for (int64_t i = 0; i < A.n; ++i)
        for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
            int32_t pos = fill[A.col[k]]++;
            T.col[pos] = (int32_t)i;
            T.val[pos] = A.val[k];
        }
    return T;
}

// Substructuring: node-plane cuts c_t = floor(t g / p), t = 1..p-1.
// Returns the number of cuts strictly below `coord` and whether coord is a cut.
static inline void axis_side(int64_t coord, int64_t g, int64_t p, int64_t& below, bool& on)
{
    below = 0;
    on = false;
    for (int64_t t = 1; t < p; ++t) {
        int64_t c = (t * g) / p;
        if (c < coord) ++below;
        else if (c == coord) on = true;
    }
}

Error make_plan(const HostCSR& A, jac_splitting s, int32_t nparts, const jac_opts& o, Plan& plan)
{
    const int64_t n = A.n;
    plan = Plan();
    plan.splitting = s;
    plan.perm.resize(n);
    plan.iperm.resize(n);
    if (s == JAC_BANDROW || s == JAC_BANDROW_NNZ) {
        if (nparts < 1 || nparts > n) return Error(JAC_EINVAL, fmt("nparts must be in [1, n=%lld]", n));
        const int64_t P = nparts;
        plan.part_ptr.resize(P + 1);
        if (s == JAC_BANDROW) {
            for (int64_t p = 0; p <= P; ++p) plan.part_ptr[p] = (p * n) / P;
        } else {
            // first row r with P * IA(r) >= k * nnz (IA non-decreasing -> lower bound)
            const int64_t nnz = A.nnz();
            for (int64_t k = 0; k <= P; ++k) {
                const int64_t target = k * nnz;
                int64_t lo = 0, hi = n;
                while (lo < hi) {
                    int64_t mid = lo + (hi - lo) / 2;
                    if (P * (int64_t)A.rowptr[mid] >= target) hi = mid;
                    else lo = mid + 1;
                }
                plan.part_ptr[k] = lo;
            }
            plan.part_ptr[0] = 0;
            plan.part_ptr[P] = n;
        }
        std::iota(plan.perm.begin(), plan.perm.end(), 0);
        std::iota(plan.iperm.begin(), plan.iperm.end(), 0);
        return Error();
    }
    if (s != JAC_SUBSTRUCT) return Error(JAC_EINVAL, "unknown splitting");
    const int64_t gx = o.grid[0], gy = o.grid[1], gz = o.grid[2];
    const int64_t px = o.subdomains[0], py = o.subdomains[1], pz = o.subdomains[2];
    if (gx < 1 || gy < 1 || gz < 1) return Error(JAC_EINVAL, "SUBSTRUCT needs opts.grid (gx, gy, gz) >= 1");
    if (px < 1 || py < 1 || pz < 1 || px > gx || py > gy || pz > gz)
        return Error(JAC_EINVAL, "SUBSTRUCT needs 1 <= opts.subdomains[d] <= grid[d]");
    const int64_t G = gx * gy * gz;
    if (!o.node_of_row && n != G) return Error(JAC_EINVAL, "n != gx*gy*gz and no node_of_row given");
    if (o.node_of_row) {
        std::vector<uint8_t> seen(G, 0);
        for (int64_t r = 0; r < n; ++r) {
            int64_t v = o.node_of_row[r];
            if (v < 0 || v >= G) return Error(JAC_EINVAL, fmt("node_of_row[%lld] outside the grid", r));
            if (seen[v]) return Error(JAC_EINVAL, fmt("node_of_row repeats node %lld", v));
            seen[v] = 1;
        }
    }
    const int64_t S = px * py * pz;
    std::vector<int64_t> sid(n);
    // precompute per-axis tables
    std::vector<int64_t> bx(gx), by(gy), bz(gz);
    std::vector<uint8_t> ox(gx), oy(gy), oz(gz);
    for (int64_t v = 0; v < gx; ++v) { bool on; axis_side(v, gx, px, bx[v], on); ox[v] = on; }
    for (int64_t v = 0; v < gy; ++v) { bool on; axis_side(v, gy, py, by[v], on); oy[v] = on; }
    for (int64_t v = 0; v < gz; ++v) { bool on; axis_side(v, gz, pz, bz[v], on); oz[v] = on; }
    for (int64_t r = 0; r < n; ++r) {
        const int64_t node = o.node_of_row ? o.node_of_row[r] : r;
        const int64_t X = node % gx, Y = (node / gx) % gy, Z = node / (gx * gy);
        sid[r] = (ox[X] || oy[Y] || oz[Z]) ? S : bx[X] + px * (by[Y] + py * bz[Z]);
    }
    plan.part_ptr.assign(S + 2, 0);
    for (int64_t r = 0; r < n; ++r) plan.part_ptr[sid[r] + 1]++;
    for (int64_t p = 0; p <= S; ++p) plan.part_ptr[p + 1] += plan.part_ptr[p];
    std::vector<int64_t> fill(plan.part_ptr.begin(), plan.part_ptr.end() - 1);
    for (int64_t r = 0; r < n; ++r) {
        int64_t pos = fill[sid[r]]++;
        plan.perm[pos] = r;
        plan.iperm[r] = pos;
    }
    plan.interface_rows = plan.part_ptr[S + 1] - plan.part_ptr[S];
    // The block form of Eq. (4.4) needs A_ij = 0 between different interiors.
    for (int64_t i = 0; i < n; ++i) {
        if (sid[i] == S) continue;
        for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
            int64_t sj = sid[A.col[k]];
            if (sj != S && sj != sid[i])
                return Error(JAC_EINVAL, fmt("subdomain interiors %lld and %lld are coupled (row %lld): "
                                             "grid/subdomains do not match the matrix", sid[i], sj, i));
        }
    }
    return Error();
}

// Stopping on local convergence (Sec. 3, the parallel form of Algorithm 1):
// the rows each partition tests.  Band splittings: band p holds its rows.
// Substructuring: subdomain s holds the nodes of its box of grid cells; along
// an axis the box t covers the closed node range [c_t, c_{t+1}] (c_0 = 0,
// c_p = g - 1 at the grid's ends), so a node on cut plane c_t belongs to the
// boxes t-1 and t, and an interface node to 2, 4 or 8 subdomains.
Error local_row_sets(const Plan& plan, const jac_opts& o, std::vector<int32_t>& mem_ptr,
                     std::vector<int32_t>& mem_part, std::vector<int32_t>& mem_head, std::vector<int32_t>& set_id)
{
    const int64_t n = (int64_t)plan.perm.size();
    std::vector<int64_t> first(n + 1, 0);        // per new row: its sets (partition numbers)
    std::vector<int64_t> parts;
    parts.reserve(n + n / 8);
    int64_t nparts = 0;
    if (plan.splitting == JAC_BANDROW || plan.splitting == JAC_BANDROW_NNZ) {
        nparts = plan.nparts();
        for (int64_t p = 0; p < nparts; ++p)
            for (int64_t r = plan.part_ptr[p]; r < plan.part_ptr[p + 1]; ++r) {
                parts.push_back(p);
                first[r + 1] = (int64_t)parts.size();
            }
    } else if (plan.splitting == JAC_SUBSTRUCT) {
        const int64_t gx = o.grid[0], gy = o.grid[1], gz = o.grid[2];
        const int64_t px = o.subdomains[0], py = o.subdomains[1], pz = o.subdomains[2];
        nparts = px * py * pz;
        // boxes of each coordinate along each axis (one, or two on a cut plane)
        auto axis_boxes = [](int64_t g, int64_t p, std::vector<int64_t>& lo, std::vector<int64_t>& cnt) {
            lo.assign(g, 0);
            cnt.assign(g, 1);
            for (int64_t v = 0; v < g; ++v) {
                int64_t below = 0;
                bool on = false;
                axis_side(v, g, p, below, on);
                lo[v] = below;                  // a cut c_t = v (t = below + 1) joins boxes below, below + 1
                cnt[v] = on ? 2 : 1;
            }
        };
        std::vector<int64_t> lx, ly, lz, cx, cy, cz;
        axis_boxes(gx, px, lx, cx);
        axis_boxes(gy, py, ly, cy);
        axis_boxes(gz, pz, lz, cz);
        for (int64_t r = 0; r < n; ++r) {
            const int64_t i = plan.perm[r];
            const int64_t node = o.node_of_row ? o.node_of_row[i] : i;
            const int64_t X = node % gx, Y = (node / gx) % gy, Z = node / (gx * gy);
            for (int64_t a = 0; a < cz[Z]; ++a)
                for (int64_t bb = 0; bb < cy[Y]; ++bb)
                    for (int64_t q = 0; q < cx[X]; ++q)
                        parts.push_back((lx[X] + q) + px * ((ly[Y] + bb) + py * (lz[Z] + a)));
            first[r + 1] = (int64_t)parts.size();
        }
    } else {
        return Error(JAC_EINVAL, "local stopping needs a band or substructuring splitting");
    }
    if ((int64_t)parts.size() > INT32_MAX - 64) return Error(JAC_EINVAL, "too many local set entries");
    // number the non-empty sets densely, in partition order
    std::vector<int32_t> dense(nparts, -1);
    for (int64_t p : parts) dense[p] = 0;
    set_id.clear();
    for (int64_t p = 0; p < nparts; ++p)
        if (dense[p] == 0) {
            dense[p] = (int32_t)set_id.size();
            set_id.push_back((int32_t)p);
        }
    if (set_id.size() >= ((size_t)1 << 24)) return Error(JAC_EINVAL, "local stopping: more than 2^24 partitions");
    mem_ptr.resize(n + 1);
    for (int64_t r = 0; r <= n; ++r) mem_ptr[r] = (int32_t)first[r];
    mem_part.resize(parts.size());
    for (size_t e = 0; e < parts.size(); ++e) mem_part[e] = dense[parts[e]];
    // per row: its first set (low 24 bits) and its number of sets (high 8 bits)
    mem_head.resize(n);
    for (int64_t r = 0; r < n; ++r) {
        const int64_t cnt = first[r + 1] - first[r];
        mem_head[r] = cnt > 0 ? (int32_t)(((uint32_t)cnt << 24) | (uint32_t)dense[parts[first[r]]]) : -1;
    }
    return Error();
}

Error make_scaled_form(const HostCSR& A, const Plan& plan, ScaledForm& tf)
{
    const int64_t n = A.n;
    tf = ScaledForm();
    tf.n = n;
    tf.rowptr.resize(n + 1);
    tf.d.resize(n);
    tf.rowptr[0] = 0;
    // pass 1: diagonal and off-diagonal counts
    for (int64_t r = 0; r < n; ++r) {
        const int64_t i = plan.perm[r];
        int ndiag = 0;
        double di = 0.0;
        int64_t off = 0;
        for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
            if (A.col[k] == i) { ++ndiag; di = A.val[k]; }
            else ++off;
        }
        if (ndiag > 1) return Error(JAC_EINVAL, fmt("row %lld stores its diagonal %lld times", i, ndiag));
        if (ndiag == 0 || di == 0.0) return Error(JAC_ESINGULAR, fmt("zero or missing diagonal in row %lld", i));
        tf.d[r] = di;
        tf.rowptr[r + 1] = (int32_t)(tf.rowptr[r] + off);
        tf.max_off = std::max(tf.max_off, off);
    }
    const int64_t nnz_off = tf.rowptr[n];
    tf.col.resize(nnz_off);
    tf.S.resize(nnz_off);
    for (int64_t r = 0; r < n; ++r) {
        const int64_t i = plan.perm[r];
        int64_t w = tf.rowptr[r];
        for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
            if (A.col[k] == i) continue;
            const int64_t rj = plan.iperm[A.col[k]];
            tf.col[w] = (int32_t)rj;
            tf.S[w] = -(A.val[k] / tf.d[rj]);     // column scaling: -a_ij / a_jj
            ++w;
        }
    }
    return Error();
}

void dependency_lists(const HostCSR& A, const Plan& plan, std::vector<int64_t>& recv_ptr,
                      std::vector<int32_t>& recv_from, std::vector<int64_t>& recv)
{
    const int64_t n = A.n, P = plan.nparts();
    std::vector<int32_t> owner(n);
    for (int64_t p = 0; p < P; ++p)
        for (int64_t r = plan.part_ptr[p]; r < plan.part_ptr[p + 1]; ++r) owner[plan.perm[r]] = (int32_t)p;
    std::vector<int64_t> stamp(n, -1);
    recv_ptr.assign(P + 1, 0);
    recv_from.clear();
    recv.clear();
    std::vector<std::pair<int32_t, int64_t>> ext;
    for (int64_t p = 0; p < P; ++p) {
        ext.clear();
        for (int64_t r = plan.part_ptr[p]; r < plan.part_ptr[p + 1]; ++r) {
            const int64_t i = plan.perm[r];
            for (int64_t k = A.rowptr[i]; k < A.rowptr[i + 1]; ++k) {
                const int64_t j = A.col[k];
                if (owner[j] != p && stamp[j] != p) {
                    stamp[j] = p;
                    ext.emplace_back(owner[j], j);
                }
            }
        }
        std::sort(ext.begin(), ext.end());
        for (auto& e : ext) { recv_from.push_back(e.first); recv.push_back(e.second); }
        recv_ptr[p + 1] = (int64_t)recv.size();
    }
}

double default_row_cost(int64_t off_entries)
{
    // Relative sweep cost of a row with `off_entries` off-diagonal entries:
    // per-row work (row length, b, own y, store, residual) weighs about as
    // much as six entries on GB300 (fitted to per-CTA times of the 160^3 sweep).
    return 6.0 + (double)off_entries;
}

double slot_row_cost(int64_t entries)
{
    // A slot row of a split interface block carries a row's fixed cost twice:
    // its own (row length, b slot, loop set-up) and its share of the in-warp
    // assembly (shuffles and adds in subdomain order, the group's store and
    // residual).  Per-CTA times of the 160^3 4x4x4 split sweep put a slot row
    // of 2 to 5 entries at about 1.3 seven-point rows.
    return 12.0 + (double)entries;
}

void make_tiling(const ScaledForm& tf, const Plan& plan, int32_t rows_per_tile, int32_t max_entries,
                 int64_t ctas, Tiling& t, const std::vector<double>* row_cost, int64_t align_from, int32_t align,
                 int64_t r_begin, int64_t r_end)
{
    auto aligned_up = [&](int64_t r) -> int64_t {
        if (align <= 1 || r <= align_from) return r;
        return std::min<int64_t>(tf.n, align_from + (r - align_from + align - 1) / align * align);
    };
    t = Tiling();
    t.rows_per_tile = rows_per_tile;
    t.max_entries = max_entries;
    const int64_t n = r_end < 0 ? tf.n : r_end;
    const int64_t b0 = r_begin;
    // CTA row ranges: contiguous, cut at row granularity so that every CTA
    // carries the same estimated cost (pre[r - b0]: cost of rows b0 .. r-1).
    std::vector<double> pre(n - b0 + 1, 0.0);
    for (int64_t r = b0; r < n; ++r) {
        const double w = row_cost ? (*row_cost)[r] : default_row_cost(tf.rowptr[r + 1] - tf.rowptr[r]);
        pre[r - b0 + 1] = pre[r - b0] + w;
    }
    std::vector<int64_t> rb(ctas + 1, b0);
    rb[ctas] = n;
    {
        int64_t cur = b0;
        const double tot = pre[n - b0];
        for (int64_t g = 1; g < ctas; ++g) {
            const double target = tot * (double)g / (double)ctas;
            while (cur < n && pre[cur - b0] + 0.5 * (pre[cur - b0 + 1] - pre[cur - b0]) < target) ++cur;
            cur = aligned_up(cur);
            rb[g] = cur;
        }
    }
    // Tiles: at most rows_per_tile rows and max_entries staged entries, never
    // crossing a partition or a CTA boundary.
    t.row0.push_back((int32_t)b0);
    t.cta0.assign(ctas + 1, 0);
    int64_t p = 0;
    const int64_t P = plan.nparts();
    for (int64_t g = 0; g < ctas; ++g) {
        t.cta0[g] = (int32_t)(t.row0.size() - 1);
        int64_t r = rb[g];
        const int64_t end = rb[g + 1];
        while (r < end) {
            while (p + 1 < P && plan.part_ptr[p + 1] <= r) ++p;
            const int64_t lim = std::min<int64_t>(end, plan.part_ptr[p + 1]);
            int64_t rows = 0, ent = 0;
            while (r + rows < lim && rows < rows_per_tile) {
                const int64_t len = tf.rowptr[r + rows + 1] - tf.rowptr[r + rows];
                if (rows > 0 && ent + len > max_entries) break;
                ent += len;
                ++rows;
                if (ent > max_entries) break;   // a single oversized row forms its own tile
            }
            if (align > 1 && r >= align_from && r + rows < lim && (r + rows - align_from) % align) {
                // aligned cut: back to the previous boundary, or on to the next one
                // (the tile then exceeds the staged entries and is read from L2)
                const int64_t down = (r + rows - align_from) / align * align + align_from;
                rows = down > r ? down - r : std::min<int64_t>(lim, aligned_up(r + rows)) - r;
            }
            r += rows;
            t.row0.push_back((int32_t)r);
            t.tile_part.push_back((int32_t)p);
        }
    }
    const int64_t nt = t.ntiles();
    t.cta0[ctas] = (int32_t)nt;
    t.nnz0.resize(nt + 1);
    for (int64_t i = 0; i <= nt; ++i) t.nnz0[i] = tf.rowptr[t.row0[i]];
}

void make_split_tiling(const SplitForm& f, int32_t rows_per_tile, int32_t max_entries, int64_t ctas, Tiling& t,
                       const std::vector<double>* row_cost)
{
    // Every CTA gets a row range of the interiors (cta0) and one of the slot
    // rows (cta1, cut on warp boundaries), so each SM runs the same mix of
    // complete rows and slot rows.  With the slot rows in the last CTAs alone,
    // those CTAs' latency-bound tiles left the SM's FP64 pipe to their
    // SM-mates, and no per-CTA cut could balance the sweep.
    Tiling t2;
    make_tiling(f.tf, f.plan, rows_per_tile, max_entries, ctas, t, row_cost, INT64_MAX, 1, 0, f.n_own);
    make_tiling(f.tf, f.plan, rows_per_tile, max_entries, ctas, t2, row_cost, f.n_own, f.warp_rows, f.n_own,
                f.tf.n);
    const int32_t T1 = (int32_t)t.ntiles();
    t.row0.insert(t.row0.end(), t2.row0.begin() + 1, t2.row0.end());
    t.nnz0.insert(t.nnz0.end(), t2.nnz0.begin() + 1, t2.nnz0.end());
    t.tile_part.insert(t.tile_part.end(), t2.tile_part.begin(), t2.tile_part.end());
    t.cta1 = t2.cta0;
    for (int32_t& v : t.cta1) v += T1;
}

void make_windows(const ScaledForm& tf, const Tiling& t, int32_t xcap, int32_t maxruns, int32_t emax, Windows& w)
{
    const int64_t nt = t.ntiles();
    const int64_t GAP = 16;     // columns closer than this join one run
    w = Windows();
    w.xcap = xcap;
    w.maxruns = maxruns;
    w.blk0.resize(nt + 1);
    w.lcol.assign(tf.col.size(), 0);
    std::vector<int32_t> cols;
    struct Run { int64_t s, e; };   // [s, e) aligned to 4
    std::vector<Run> runs;
    for (int64_t ti = 0; ti < nt; ++ti) {
        const int64_t r0 = t.row0[ti], r1 = t.row0[ti + 1];
        const int64_t p0 = tf.rowptr[r0], p1 = tf.rowptr[r1];
        w.blk0[ti] = (int32_t)(w.blk.size() / 4);
        cols.assign(tf.col.begin() + p0, tf.col.begin() + p1);
        for (int64_t r = r0; r < r1; ++r) cols.push_back((int32_t)r);
        std::sort(cols.begin(), cols.end());
        cols.erase(std::unique(cols.begin(), cols.end()), cols.end());
        runs.clear();
        for (int32_t c : cols) {
            const int64_t a = (int64_t)c & ~(int64_t)3;
            if (!runs.empty() && a <= runs.back().e + GAP) {
                runs.back().e = std::max<int64_t>(runs.back().e, ((int64_t)c + 4) & ~(int64_t)3);
            } else {
                runs.push_back({a, ((int64_t)c + 4) & ~(int64_t)3});
            }
        }
        int64_t xlen = 0;
        for (auto& rn : runs) xlen += rn.e - rn.s;
        const bool fb = (p1 - p0) > emax || xlen > xcap || (int64_t)runs.size() > maxruns;
        int64_t own = 0;
        if (!fb) {
            int64_t off = 0;
            for (auto& rn : runs) {
                if (r0 >= rn.s && r0 < rn.e) own = off + (r0 - rn.s);
                off += rn.e - rn.s;
            }
            // local column of every entry: offset of its run + position in the run
            for (int64_t k = p0; k < p1; ++k) {
                const int64_t c = tf.col[k];
                int64_t lo = 0, hi = (int64_t)runs.size() - 1, o2 = 0;
                while (lo < hi) {               // last run with s <= c
                    int64_t mid = (lo + hi + 1) / 2;
                    if (runs[mid].s <= c) lo = mid;
                    else hi = mid - 1;
                }
                for (int64_t q = 0; q < lo; ++q) o2 += runs[q].e - runs[q].s;
                w.lcol[k] = (int32_t)(o2 + (c - runs[lo].s));
            }
            w.window_elems += xlen;
        } else {
            ++w.fallback_tiles;
        }
        const int32_t nr = fb ? 0 : (int32_t)runs.size();
        w.blk.insert(w.blk.end(), {(int32_t)(fb ? 0 : xlen), (int32_t)own, nr, fb ? TILE_FALLBACK : 0});
        int64_t dst = 0;
        for (int32_t q = 0; q < nr; ++q) {
            w.blk.insert(w.blk.end(), {(int32_t)runs[q].s, (int32_t)(runs[q].e - runs[q].s), (int32_t)dst, 0});
            dst += runs[q].e - runs[q].s;
        }
    }
    w.blk0[nt] = (int32_t)(w.blk.size() / 4);
}

// ---------------------------------------------------------------- split interface

int32_t split_max_multiplicity(int64_t n, int32_t nsub, const jac_local* sub)
{
    if (n < 1 || nsub < 1 || !sub) return 0;
    std::vector<int32_t> mult(n, 0);
    int32_t mx = 0;
    for (int32_t s = 0; s < nsub; ++s) {
        if (sub[s].n < 0 || (sub[s].n > 0 && !sub[s].l2g)) return 0;
        for (int32_t l = 0; l < sub[s].n; ++l) {
            const int64_t g = sub[s].l2g[l];
            if (g < 0 || g >= n) return 0;
            mx = std::max(mx, ++mult[g]);
        }
    }
    return mx;
}

Error make_split_form(int64_t n, int32_t nsub, const jac_local* sub, int32_t warp_rows, SplitForm& out)
{
    out = SplitForm();
    if (n < 1) return Error(JAC_EINVAL, "n must be >= 1");
    if (n > INT32_MAX - 64) return Error(JAC_EINVAL, "n too large");
    if (nsub < 1 || nsub > 65536) return Error(JAC_EINVAL, "nsub must be in 1..65536");
    if (!sub) return Error(JAC_EINVAL, "sub is NULL");
    if (warp_rows < 1 || warp_rows > 32) return Error(JAC_EINVAL, "bad warp_rows");
    // ---- validate each local matrix; multiplicities; diagonals
    std::vector<int32_t> mult(n, 0), stamp(n, -1);
    std::vector<double> d(n, 0.0);
    int64_t nnz_all = 0;
    for (int32_t s = 0; s < nsub; ++s) {
        const jac_local& L = sub[s];
        char msg[160];
        if (L.n < 0 || L.nnz < 0) {
            std::snprintf(msg, sizeof(msg), "subdomain %d: negative size", s);
            return Error(JAC_EINVAL, msg);
        }
        if (L.n == 0) continue;
        if (!L.rowptr || !L.l2g || (L.nnz > 0 && (!L.col || !L.val))) {
            std::snprintf(msg, sizeof(msg), "subdomain %d: NULL array", s);
            return Error(JAC_EINVAL, msg);
        }
        if (L.rowptr[0] != 0 || L.rowptr[L.n] != L.nnz) {
            std::snprintf(msg, sizeof(msg), "subdomain %d: rowptr must run from 0 to nnz", s);
            return Error(JAC_EINVAL, msg);
        }
        nnz_all += L.nnz;
        if (nnz_all >= INT32_MAX) return Error(JAC_EINVAL, "total local nnz >= 2^31");
        for (int32_t l = 0; l < L.n; ++l) {
            const int64_t g = L.l2g[l];
            if (g < 0 || g >= n) {
                std::snprintf(msg, sizeof(msg), "subdomain %d: l2g[%d] = %lld out of range", s, l, (long long)g);
                return Error(JAC_EINVAL, msg);
            }
            if (stamp[g] == s) {
                std::snprintf(msg, sizeof(msg), "subdomain %d: row %lld listed twice in l2g", s, (long long)g);
                return Error(JAC_EINVAL, msg);
            }
            stamp[g] = s;
            ++mult[g];
            if (L.rowptr[l + 1] < L.rowptr[l]) {
                std::snprintf(msg, sizeof(msg), "subdomain %d: rowptr decreases at %d", s, l);
                return Error(JAC_EINVAL, msg);
            }
            int ndiag = 0;
            for (int64_t k = L.rowptr[l]; k < L.rowptr[l + 1]; ++k) {
                if (L.col[k] < 0 || L.col[k] >= L.n) {
                    std::snprintf(msg, sizeof(msg), "subdomain %d: column index out of range in local row %d", s, l);
                    return Error(JAC_EINVAL, msg);
                }
                if (L.col[k] == l) {
                    if (++ndiag > 1) {
                        std::snprintf(msg, sizeof(msg), "subdomain %d: two diagonal entries in local row %d", s, l);
                        return Error(JAC_EINVAL, msg);
                    }
                    d[g] += L.val[k];         // subdomains in ascending order
                }
            }
        }
    }
    int32_t max_mult = 0;
    for (int64_t g = 0; g < n; ++g) {
        if (mult[g] == 0) {
            char msg[96];
            std::snprintf(msg, sizeof(msg), "row %lld belongs to no subdomain", (long long)g);
            return Error(JAC_EINVAL, msg);
        }
        if (d[g] == 0.0 || !std::isfinite(d[g])) {
            char msg[96];
            std::snprintf(msg, sizeof(msg), "assembled diagonal of row %lld is %g", (long long)g, d[g]);
            return Error(JAC_ESINGULAR, msg);
        }
        max_mult = std::max(max_mult, mult[g]);
    }
    if (max_mult > warp_rows) {
        char msg[128];
        std::snprintf(msg, sizeof(msg), "a row is held by %d subdomains; at most %d with %d lanes per row", max_mult,
                      warp_rows, 32 / warp_rows);
        return Error(JAC_EINVAL, msg);
    }
    // ---- holders of every row, ascending subdomain: (s, local row)
    std::vector<int64_t> hptr(n + 1, 0);
    for (int64_t g = 0; g < n; ++g) hptr[g + 1] = hptr[g] + mult[g];
    std::vector<int32_t> hsub(hptr[n]), hloc(hptr[n]);
    {
        std::vector<int64_t> fill(hptr.begin(), hptr.end() - 1);
        for (int32_t s = 0; s < nsub; ++s)
            for (int32_t l = 0; l < sub[s].n; ++l) {
                const int64_t g = sub[s].l2g[l];
                hsub[fill[g]] = s;
                hloc[fill[g]++] = l;
            }
    }
    // ---- new order: interiors by subdomain (ascending row), then the interface
    Plan& P = out.plan;
    P.splitting = JAC_SUBSTRUCT;
    P.perm.reserve(n);
    std::vector<int64_t> cnt(nsub + 1, 0);
    for (int64_t g = 0; g < n; ++g)
        if (mult[g] == 1) ++cnt[hsub[hptr[g]] + 1];
    for (int32_t s = 0; s < nsub; ++s) cnt[s + 1] += cnt[s];
    const int64_t n_own = cnt[nsub];
    P.perm.assign(n, -1);
    {
        std::vector<int64_t> fill(cnt.begin(), cnt.end() - 1);
        int64_t f = n_own;
        for (int64_t g = 0; g < n; ++g) {
            if (mult[g] == 1) P.perm[fill[hsub[hptr[g]]]++] = g;
            else P.perm[f++] = g;
        }
    }
    P.iperm.assign(n, 0);
    for (int64_t r = 0; r < n; ++r) P.iperm[P.perm[r]] = r;
    out.n = n;
    out.n_own = n_own;
    out.n_ifc = n - n_own;
    out.nnz_local = nnz_all;
    out.warp_rows = warp_rows;
    out.max_mult = max_mult;
    if (out.n_ifc >= (int64_t)1 << 26) return Error(JAC_EINVAL, "interface too large (>= 2^26 rows)");
    // ---- kernel rows
    ScaledForm& tf = out.tf;
    tf.d.resize(n);
    for (int64_t r = 0; r < n; ++r) tf.d[r] = d[P.perm[r]];
    tf.rowptr.assign(1, 0);
    auto push_row = [&](int32_t s, int32_t l) {
        const jac_local& L = sub[s];
        for (int64_t k = L.rowptr[l]; k < L.rowptr[l + 1]; ++k) {
            if (L.col[k] == l) continue;
            const int64_t gj = L.l2g[L.col[k]];
            tf.col.push_back((int32_t)P.iperm[gj]);
            tf.S.push_back(-L.val[k] / d[gj]);
        }
        const int64_t len = (int64_t)tf.col.size() - tf.rowptr.back();
        tf.max_off = std::max(tf.max_off, len);
        if ((int64_t)tf.col.size() >= INT32_MAX) return false;
        tf.rowptr.push_back((int32_t)tf.col.size());
        return true;
    };
    out.bmap.reserve(n + (size_t)out.n_ifc * 2);
    for (int64_t r = 0; r < n_own; ++r) {
        const int64_t g = P.perm[r];
        if (!push_row(hsub[hptr[g]], hloc[hptr[g]])) return Error(JAC_EINVAL, "too many entries");
        out.bmap.push_back(g);
    }
    P.part_ptr.assign(cnt.begin(), cnt.end());     // subdomain interiors
    int64_t pos = 0;                                // slot rows after n_own
    auto pad_row = [&]() {
        tf.rowptr.push_back(tf.rowptr.back());
        out.bmap.push_back(-1);
        out.slot_info.push_back(0u);
        ++pos;
    };
    for (int64_t i = 0; i < out.n_ifc; ++i) {
        const int64_t g = P.perm[n_own + i];
        const int32_t m = mult[g];
        if (pos % warp_rows + m > warp_rows)
            while (pos % warp_rows) pad_row();
        for (int32_t q = 0; q < m; ++q) {
            if (!push_row(hsub[hptr[g] + q], hloc[hptr[g] + q])) return Error(JAC_EINVAL, "too many entries");
            out.bmap.push_back(q == 0 ? g : -1);
            out.slot_info.push_back(q == 0 ? ((uint32_t)i << 6) | (uint32_t)m : 0u);
            ++pos;
        }
        out.partials += m;
    }
    tf.n = n_own + pos;
    if (tf.n > INT32_MAX - 64) return Error(JAC_EINVAL, "too many kernel rows");
    P.part_ptr.push_back(tf.n);                    // the interface partition
    P.interface_rows = out.n_ifc;
    return Error();
}

}  // namespace jac
