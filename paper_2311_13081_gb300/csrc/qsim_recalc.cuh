// qsim_recalc.cuh -- reward recalculation of stored transitions (Sec. VI: after each
// change of the reward constants every reward in the replay buffer is recomputed from the
// stored successor state and action), shared by the stand-alone kernel and the training
// kernel's curriculum step.
#pragma once
#include "qsim_internal.h"

namespace qsim {

__device__ __forceinline__ float4 ld4s(const float* p, int q) { return __ldcs(reinterpret_cast<const float4*>(p) + q); }

__device__ __forceinline__ float comp(const float4& v, int j) {
    return j == 0 ? v.x : (j == 1 ? v.y : (j == 2 ? v.z : v.w));
}

// Recomputes r of envs 4q .. 4q+3 in ring slot `slot`.  s' is the side slot where the
// episode ended (flag bits 0-1), the next slot's s otherwise, or the live state when the
// record is the newest one.  One float4 load per field across the four envs (streaming:
// each value is read once); the side slot is read only when one of the four episodes
// ended.  The record layout is [slot][field][ld] with ld a multiple of 4.
__device__ __forceinline__ void recalc_quad(const EnvCfg& C, const EnvPtrs& p, const float* Cr,
                                            int64_t slot, int64_t next, bool newest, int q) {
    const size_t ld = (size_t)C.ld;
    float* rec = p.rec + (size_t)slot * (size_t)C.F * ld;
    const uint4 fl = __ldcs(reinterpret_cast<const uint4*>(rec + 22 * ld) + q);
    float4 a[4], s2[NS];
#pragma unroll
    for (int i = 0; i < 4; ++i) a[i] = ld4s(rec + (17 + i) * ld, q);
    const float* src = newest ? p.state : p.rec + (size_t)next * (size_t)C.F * ld;
#pragma unroll
    for (int i = 0; i < NS; ++i) s2[i] = ld4s(src + i * ld, q);
    const bool d0 = (fl.x & 3u) != 0, d1 = (fl.y & 3u) != 0, d2 = (fl.z & 3u) != 0, d3 = (fl.w & 3u) != 0;
    if (d0 || d1 || d2 || d3) {
        // env-major side slot: the 17 values of an ended env are contiguous (68 B), read only
        // for the envs whose episode ended
        const float* sd = p.side + ((size_t)slot * ld + 4 * (size_t)q) * NS;
        const bool dj[4] = {d0, d1, d2, d3};
#pragma unroll
        for (int j = 0; j < 4; ++j) {
            if (!dj[j]) continue;
            float x[NS];
#pragma unroll
            for (int i = 0; i < NS; ++i) x[i] = __ldcs(sd + j * NS + i);
#pragma unroll
            for (int i = 0; i < NS; ++i) {
                if (j == 0) s2[i].x = x[i];
                else if (j == 1) s2[i].y = x[i];
                else if (j == 2) s2[i].z = x[i];
                else s2[i].w = x[i];
            }
        }
    }
    float r[4];
#pragma unroll
    for (int j = 0; j < 4; ++j) {
        float s[NS], aa[4];
#pragma unroll
        for (int i = 0; i < NS; ++i) s[i] = comp(s2[i], j);
#pragma unroll
        for (int i = 0; i < 4; ++i) aa[i] = comp(a[i], j);
        r[j] = reward(Cr, s, aa);
    }
    __stcs(reinterpret_cast<float4*>(rec + 21 * ld) + q, make_float4(r[0], r[1], r[2], r[3]));
}

// Quads [i0, size * ceil(n / 4)) with stride `step` of the ring holding `size` records
// ending at `head` (exclusive): k-major, so consecutive threads take consecutive quads of a
// slot (the last quad may reach into the padding up to ld, whose r is unspecified).  The
// quad count is < 2^32 (the callers check), so the index splits with one 32-bit division.
__device__ __forceinline__ void recalc_range(const EnvCfg& C, const EnvPtrs& p, const float* Cr, int64_t head,
                                             int64_t size, int64_t capacity, uint64_t i0, uint64_t step) {
    const uint32_t Q = ((uint32_t)C.n + 3u) >> 2;
    const uint64_t total = (uint64_t)size * Q;
    for (uint64_t i = i0; i < total; i += step) {
        const uint32_t k = (uint32_t)i / Q, q = (uint32_t)i - k * Q;
        int64_t slot = head - size + (int64_t)k;  // in [-capacity, capacity)
        if (slot < 0) slot += capacity;
        const int64_t next = slot + 1 == capacity ? 0 : slot + 1;
        const bool newest = (int64_t)k == size - 1;
        // (debug builds) slots and the env quad checked against the allocation
        if (!in_bounds(p.status, slot, p.rows, SITE_RING_READ) ||
            (!newest && !in_bounds(p.status, next, p.rows, SITE_RING_READ)) ||
            !in_bounds(p.status, 4 * (int64_t)q + 3, C.ld, SITE_SOA))
            continue;
        recalc_quad(C, p, Cr, slot, next, newest, (int)q);
    }
}

}  // namespace qsim
