// Launch arguments and entry points of the 2-opt local search (Sec. 5.7),
// kept apart from the construction / pheromone declarations.
#pragma once

#include "internal.cuh"

namespace mmas {

struct TwoOptArgs {
    int32_t n, m, ld, k;
    const int32_t *nn;     // [n][k] neighbour lists (the candidate lists)
    const uint16_t *nn16;  // the same lists as 16-bit ids (padded to 16 bytes)
    const int32_t *nnd;    // [n][k] distance to each neighbour
    const int2 *xy;        // coordinates, or nullptr (then dist)
    const int32_t *dist;   // [n][ld]
    int32_t *tours;        // [m][ld], improved in place
    int32_t *lens;         // [m]: read (iteration best) and written
    uint32_t *err;         // device error bits
};

// Dynamic shared memory of one 2-opt CTA for an n-city tour with k
// neighbours; `staged` adds the coordinates and the 16-bit neighbour lists.
size_t two_opt_smem(int n, int k, bool staged);
// Whether the dynamic layout plus the kernel's static shared memory (under
// 2 KB) fits in `smem_optin` bytes.
bool two_opt_fits(int n, int k, bool staged, size_t smem_optin);
cudaError_t launch_two_opt(const TwoOptArgs &a, bool iteration_best, int num_sms, int smem_optin,
                           cudaStream_t s);
cudaError_t launch_neighbour_dist(const TwoOptArgs &a, int32_t *nnd, cudaStream_t s);
// Testing aid: the move cap of the 2-opt search on the current device
// (cap <= 0: the default 64 n).
cudaError_t set_two_opt_move_cap(long long cap);

}  // namespace mmas
