// backtrack.cuh -- the backtracking walk of Eq. 12 for one unit, shared by the backtrack kernel and the
// fused recursion+backtrack variant of the recursion kernel.
#pragma once

#include "hgm_internal.cuh"

namespace hgm {

// From the initial pair (z_1, z_2) of Eq. 13 follow z_i = beta_i(z_{i-1}, z_{i-2}) through the unit's byte
// tables ub ([(M-2) x K x K], row (i-2)*K + slot(z_{i-1}), column slot(z_{i-2})); slots map to sorted scene
// indices through the candidate lists cidx ([M x K]) and then to the caller's indices, written in the
// caller's model order. Infeasible units (z1 < 0) get a row of -1; energy is written as given.
__device__ __forceinline__ void backtrack_unit(const Unit &un, const ModelRec &md, const SceneRec &sc, int K,
                                               const int32_t *cidx, const uint8_t *ub, const UnitResult &r,
                                               float *energy, int32_t *assign)
{
    const int M = md.M;
    if (energy) energy[un.out_e] = r.energy;
    if (!assign) return;
    int32_t *out = assign + un.out_a;
    if (r.z1 < 0) {
        for (int i = 0; i < M; ++i) out[i] = -1;
        return;
    }
    int s2 = r.z1, s1 = r.z2;   // slots of z_{i-2}, z_{i-1}
    out[md.perm[0]] = sc.perm[cidx[s2]];
    out[md.perm[1]] = sc.perm[cidx[K + s1]];
    bool ok = true;
    for (int i = 2; i < M; ++i) {
        const int s0 = ok ? ub[((int64_t)(i - 2) * K + s1) * K + s2] : kNoSlot;
        if (s0 == kNoSlot) {
            ok = false;
            out[md.perm[i]] = -1;
            continue;
        }
        out[md.perm[i]] = sc.perm[cidx[(int64_t)i * K + s0]];
        s2 = s1;
        s1 = s0;
    }
}

}  // namespace hgm
