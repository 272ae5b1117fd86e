// Host-side setup of the AMG hierarchy: CSR validation, strength of
// connection, greedy aggregation and multicolouring (Sec. 2.1).
#pragma once

#include <cstdint>
#include <string>
#include <vector>

#include "amg.h"

namespace amg {

struct HostCsr {
    int32_t n = 0;
    std::vector<int32_t> rp, ci;
    std::vector<double> va;
    int64_t nnz() const { return rp.empty() ? 0 : rp[n]; }
};

struct AggResult {
    std::vector<int32_t> agg;   // coarse index per row, -1 = not aggregated
    int32_t nc = 0;
    int32_t max_size = 0;
    int32_t n_isolated = 0;
    int32_t n_dirichlet = 0;
};

// Checks sortedness/uniqueness of columns, a positive diagonal and a
// symmetric pattern.  Returns false with a message in err.
bool validate_csr(const HostCsr& A, std::string& err);

// Algorithm 1 (with Algorithms 2, 3, the singleton merge and the isolated
// phase) on the graph of A under the parameters p.
AggResult aggregate(const HostCsr& A, const amg_params& p);

// Decoupled aggregation (Alg. 4): the rows split into consecutive tiles of
// `tile` rows, each aggregated on its own induced submatrix by `aggregate`;
// aggregates are numbered tile by tile.  Tiles run on up to `threads` host
// threads; the result does not depend on the thread count.
AggResult aggregate_tiled(const HostCsr& A, const amg_params& p, int32_t tile, int threads);

// With the environment variable AMG_CHECK set to a value other than 0:
// every stored A_ij equals A_ji exactly (the method assumes a symmetric
// matrix; validate_csr checks the pattern only).  Returns false and names the
// first offending entry otherwise.
bool check_values_symmetric(const HostCsr& A, std::string& err);

// Greedy colouring in ascending row order; returns the number of colours.
int32_t greedy_colouring(const HostCsr& A, std::vector<int32_t>& colour);

// DSATUR colouring (Brelaz): the uncoloured row with the most distinct
// colours among its neighbours next, ties to more neighbours, then to the row
// whose saturation reached its value first (initially the lower index;
// colouring a row raises its neighbours' saturations in column order);
// returns the number of colours.
int32_t dsatur_colouring(const HostCsr& A, std::vector<int32_t>& colour);

// The smoother's colouring: DSATUR when it needs fewer colours than the
// ascending-order greedy, else the greedy one.
int32_t smoother_colouring(const HostCsr& A, std::vector<int32_t>& colour);

}  // namespace amg
