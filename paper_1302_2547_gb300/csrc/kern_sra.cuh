// kern_sra.cuh -- subgraph reshaping of an aggregation (Section 3.2, Algorithm 3): the
// entry points that setup.cu calls.
#pragma once
#include "common.cuh"

namespace uaamg {

constexpr int kSraUnionMax = 16;  // largest union of a reshaped aggregate pair

// Salt of the pair weights of round `round` on level `level`.
uint32_t sra_round_salt(uint64_t seed, int level, int round);

// Rounds of Algorithm 3 on matched aggregate pairs of one level's aggregation: agg is
// updated in place, *aggptr and *members are replaced by setup temporaries holding the new
// member lists (ascending).  Runs h->p.sra_rounds rounds on the handle's stream.
int reshape_aggregation(Handle* h, int level, int n, const int* rowptr, const int* col,
                        const double* val, int nc, int* agg, int** aggptr, int** members,
                        int* scan_tmp);

}  // namespace uaamg
