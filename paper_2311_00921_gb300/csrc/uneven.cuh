// Uneven trees (leaf orders that differ, ranks min(rank, order)) embedded in the
// uniform (leaf, rank) format of the kernels (uneven.cu).
#pragma once
#include <cuda_runtime.h>

#include <vector>

#include "../../include/hss.h"

struct UnevenPad {
  long long npad = 0;           // leaf * 2^levels
  std::vector<double> D, U, E, S;   // padded generators, uniform packed layout
  std::vector<int> pmap;        // npad entries: the caller's row of each padded row, or -1
};

// Builds the padded generators of an uneven tree (shape.node_sizes set; host
// generators in the uneven packed layout of hss.h).  HSS_OK or
// HSS_ERR_INVALID_ARG (orders out of range, sizes that do not sum to n).
int pad_uneven(const hss_shape& s, const double* D, const double* U, const double* E,
               const double* S, UnevenPad* out);

// to_pad = 1: P (npad x nc, ld ldp) = the caller's rows of V (n x nc, ld ldv),
// zero on padded rows; to_pad = 0: V rows = their rows of P.
void launch_pad_rows(const double* V, int ldv, double* P, int ldp, const int* pmap, int npad,
                     int nc, int to_pad, cudaStream_t st);
