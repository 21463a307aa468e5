// Smoothed-aggregation levels (amg.cu) for use inside the step: the levels
// of a square operator whose fine pattern and FP64 value array belong to the
// caller, fed to MGHier<T> (kind 0) in place of a geometric hierarchy.
#pragma once

#include <vector>

#include "internal.h"

namespace chnss {

struct AmgHandle;

// Symbolic setup (aggregates, patterns, SELL views) of the operator with
// pattern P0 (device arrays and host copies; kept by reference) whose values
// will sit at val0 (device, read at every amg_refresh).  Synchronises s.
AmgHandle *amg_attach(const Pattern &P0, double *val0, cudaStream_t s);
// Numeric setup from the current *val0 (spectral bounds, prolongators,
// Galerkin products, transfer values) on s, without synchronisation.
void amg_refresh(AmgHandle *h, cudaStream_t s);
// The levels for MGHier<T>::init and its hi_ext.
void amg_levels(AmgHandle *h, std::vector<const Pattern *> &pats, std::vector<const int *> &diags,
                std::vector<const double *> &vals, std::vector<const Transfer *> &trs,
                std::vector<const double *> &his);
void amg_release(AmgHandle *h);

}  // namespace chnss
