// Internal declarations of the GB300 Jacobi library (host side).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "../../include/jacobi.h"

namespace jac {

// A square matrix in 0-based CSR, host memory.
struct HostCSR {
    int64_t n = 0;
    std::vector<int32_t> rowptr;   // n+1
    std::vector<int32_t> col;      // nnz
    std::vector<double> val;       // nnz
    int64_t nnz() const { return rowptr.empty() ? 0 : rowptr.back(); }
};

// Row permutation and partition ranges of a splitting (paper Sec. 4).
struct Plan {
    int32_t splitting = JAC_BANDROW;
    std::vector<int64_t> perm;      // perm[new] = original row
    std::vector<int64_t> iperm;     // iperm[original] = new row
    std::vector<int64_t> part_ptr;  // partition p owns new rows [part_ptr[p], part_ptr[p+1])
    int64_t interface_rows = 0;     // SUBSTRUCT only
    int64_t nparts() const { return (int64_t)part_ptr.size() - 1; }
};

// Off-diagonal part of P A P^T for the Jacobi iteration of Sec. 3 carried in
// the diagonally scaled iterate y = D x:
//   y'_i = b_i + sum_j S_ij y_j,  S_ij = -a_ij / a_jj   (so y' = D x' with
//   x' = D^{-1}(b - (L+U) x)),  residual r_i = y'_i - y_i,
// rows in the new order, each row's entries in the ORIGINAL stored order with
// columns renumbered to the new order.  d_i = a_ii.
struct ScaledForm {
    int64_t n = 0;
    std::vector<int32_t> rowptr;    // n+1 (off-diagonal entries only)
    std::vector<int32_t> col;       // new column indices
    std::vector<double> S;          // -a_ij / a_jj (iteration on y = D x)
    std::vector<double> d;          // a_ii (new order)
    int64_t max_off = 0;            // longest off-diagonal row
};

// Row tiles (contiguous new-row ranges that never cross a partition) and
// their assignment to CTAs.
struct Tiling {
    int32_t rows_per_tile = 256;
    int32_t max_entries = 0;            // cap of off-diagonal entries in a staged tile
    std::vector<int32_t> row0;          // ntiles+1 tile row boundaries
    std::vector<int32_t> nnz0;          // ntiles+1: off-diagonal rowptr at the boundaries
    std::vector<int32_t> cta0;          // ctas+1 tile ranges per CTA
    std::vector<int32_t> cta1;          // ctas+1: a second tile range per CTA (a split interface block's
                                        // slot tiles), empty otherwise
    std::vector<int32_t> tile_part;     // partition of each tile
    int64_t ntiles() const { return (int64_t)row0.size() - 1; }
};

// Per-tile x windows: the dependency list of a tile (Sec. 4.2.2), as a few
// contiguous runs of x that together cover every column the tile reads plus
// its own rows.  Runs start on a multiple of 4 elements and have a length that
// is a multiple of 4, so both FP64 and FP32 windows can be moved with 16-byte
// aligned bulk copies.  lcol[k] is entry k's index inside its tile's window.
// Block of a tile in `blk` (int4 units): header {xlen, own_off, nruns, flags}
// followed by nruns records {src, len, dst, 0}.
struct Windows {
    int32_t xcap = 0, maxruns = 0;
    std::vector<int32_t> blk0;          // ntiles+1, int4 offsets into blk
    std::vector<int32_t> blk;           // 4 ints per record
    std::vector<int32_t> lcol;          // nnz_off local columns (undefined on fallback tiles)
    int64_t fallback_tiles = 0;
    int64_t window_elems = 0;           // sum of window lengths (x values staged per sweep)
};
enum : int32_t { TILE_FALLBACK = 1 };   // tile reads x from L2 with global columns

// Substructuring with the interface block split between subdomains (Sec.
// 4.3), laid out for the persistent kernel.  Kernel rows: the n_own interior
// rows first (row r is iterate entry r), then "slot rows": one per (interface
// row g, subdomain s holding g), carrying the off-diagonal entries of
// (A_s)_g.  The slot rows of one interface row are consecutive, in ascending
// subdomain order, and never straddle a multiple of warp_rows (counted from
// n_own; padding rows are empty), so one warp holds all of them; the first
// one starts from b_g and its lane adds the others' sums in order.
struct SplitForm {
    ScaledForm tf;                      // tf.n = kernel rows; tf.d has the n assembled diagonals
    Plan plan;                          // perm/iperm over the n rows; part_ptr over kernel rows
    int64_t n = 0, n_own = 0, n_ifc = 0, nnz_local = 0, partials = 0;
    int32_t warp_rows = 32, max_mult = 1;
    std::vector<uint32_t> slot_info;    // per slot row: (interface index << 6) | group size at a
                                        // group's first row, 0 elsewhere
    std::vector<int64_t> bmap;          // per kernel row: original row whose b starts the sum, -1 = none
};

struct Error {
    jac_status st = JAC_OK;
    std::string msg;
    Error() = default;
    Error(jac_status s, std::string m) : st(s), msg(std::move(m)) {}
    bool ok() const { return st == JAC_OK; }
};

// jac_partition.cpp
Error host_csr_from_abi(const jac_csr* A, bool transpose, HostCSR& out);   // A must be host memory
Error make_plan(const HostCSR& A, jac_splitting s, int32_t nparts, const jac_opts& o, Plan& plan);
Error make_scaled_form(const HostCSR& A, const Plan& plan, ScaledForm& tf);
void dependency_lists(const HostCSR& A, const Plan& plan, std::vector<int64_t>& recv_ptr,
                      std::vector<int32_t>& recv_from, std::vector<int64_t>& recv);
// row_cost: per-row cost estimates in the new order (NULL: default_row_cost).
double default_row_cost(int64_t off_entries);
// Cost estimate of a slot row (split interface block), same units.
double slot_row_cost(int64_t entries);
// Rows at and after align_from are cut only at align_from + multiples of align.
// Only rows [r_begin, r_end) are tiled (r_end < 0: to the last row).
void make_tiling(const ScaledForm& tf, const Plan& plan, int32_t rows_per_tile, int32_t max_entries,
                 int64_t ctas, Tiling& t, const std::vector<double>* row_cost = nullptr,
                 int64_t align_from = INT64_MAX, int32_t align = 1, int64_t r_begin = 0, int64_t r_end = -1);
// Validates the local matrices and builds the split layout for lanes = 32 / warp_rows.
Error make_split_form(int64_t n, int32_t nsub, const jac_local* sub, int32_t warp_rows, SplitForm& out);
// Tiles of a split layout: the interiors' tiles, then the slot rows' tiles
// (on warp boundaries); each CTA owns a range of each (cta0, cta1).
void make_split_tiling(const SplitForm& f, int32_t rows_per_tile, int32_t max_entries, int64_t ctas, Tiling& t,
                       const std::vector<double>* row_cost = nullptr);
// Largest number of subdomains holding one row (0 if the input is malformed).
int32_t split_max_multiplicity(int64_t n, int32_t nsub, const jac_local* sub);
HostCSR transpose_csr(const HostCSR& A);
// Stopping on local convergence: the rows each partition holds, as a CSR
// over the new rows (mem_part: dense set numbers 0..nsets-1 of the non-empty
// sets; mem_head[r]: row r's first set | (its number of sets << 24); set_id[q]:
// the partition number of set q -- band, or subdomain sx + px (sy + py sz)).
Error local_row_sets(const Plan& plan, const jac_opts& o, std::vector<int32_t>& mem_ptr,
                     std::vector<int32_t>& mem_part, std::vector<int32_t>& mem_head, std::vector<int32_t>& set_id);
void make_windows(const ScaledForm& tf, const Tiling& t, int32_t xcap, int32_t maxruns, int32_t emax, Windows& w);

}  // namespace jac
