// Internal declarations of the vector transfers between sectors (ed_basis.cu):
// restriction to a subgroup's sector and one-site S^z sums.
#pragma once

#include "ed_internal.h"

namespace ed {
ed_status restrict_vectors(const ed_basis* from, const ed_basis* to, ed_dtype dtype, const void* x, void* y, int nvec,
                           cudaStream_t s);
ed_status sz_transfer(const ed_basis* from, const ed_basis* to, const double* c, ed_dtype dtype, const void* x, void* y,
                      int nvec, cudaStream_t s);
}  // namespace ed
