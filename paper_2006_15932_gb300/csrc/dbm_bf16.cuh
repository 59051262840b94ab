// dbm_bf16.cuh -- the BF16-deviation storage of the D2V16 state.
//
// Each cell keeps float reference moments (n^s for every species, the
// mixture u_x, u_y and T) and, per species and velocity, a bfloat16
// deviation delta, so that
//     f_i^s = f^eq_i(n^s, u, T) + delta_i^s,
// with f^eq evaluated by the FP32 symmetry-block equilibrium (feq_ref).
// The reference moments are those of the previous state, so delta is small
// (of the order of the nonequilibrium part plus one step's change) and its
// 8-bit mantissa costs far less than storing f itself in 16 bits.  Every
// reconstruction of a cell (as centre or as halo of a neighbour, in the
// step and in the output kernels) runs feq_ref on the same stored values.
#pragma once
#include <cuda_bf16.h>

#include "dbm_step_impl.cuh"

namespace dbm {

// Reference equilibrium of species s at stored (n, u, T), FP32, for one
// cell (V = float) or two (V = float2, bit for bit the same per cell).
template <int S, class V>
__device__ __forceinline__ void feq_ref(const StepConsts<float, S> &k, int s, V n, V ux, V uy, V T, V f[Q])
{
    V c[16], o[16];
    fhat_blocks<V>(n, ux, uy, vmul(T, bc<V>(k.inv_m[s])), k.dpi[s], c);
    solve_blocks<V>(k, s, c, o);
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] = feq_of<V>(i, o);
}

// Pointers of one BF16-deviation state buffer.
struct BfState {
    __nv_bfloat16 *d;  // 16 S deviation planes
    float *mom;        // S + 3 moment planes: n^0..n^{S-1}, u_x, u_y, T
    long long P;       // elements per plane
};

// Output policy of the step: delta^{n+1} = f^{n+1} - f^eq(moments of f^n)
// (the collision equilibrium the step has just built) and those moments, for
// one cell or for the pair (x, y), (x + 1, y) (x even: the pair's bfloat16
// values are one 4-byte store, its floats one 8-byte store).  No ghost
// cells: the step rebuilds a boundary tile's halo from the source cells
// (periodic wrap or outflow edge).
struct BfOut {
    static constexpr bool kNoImages = true;
    BfState st;
    int S;
    unsigned *flag;  // checked builds: where an out-of-range index is reported
    __device__ __forceinline__ void put(const Site &w, int p, float g, float e) const
    {
        const long long i = (long long)p * st.P + w.cell;
        if (in_bounds(i, 16LL * S * st.P, flag)) __stcs(st.d + i, __float2bfloat16_rn(g - e));
    }
    __device__ __forceinline__ void put(const Site &w, int p, float2 g, float2 e) const
    {
        const long long i = (long long)p * st.P + w.cell;
        if (!in_bounds(i, 16LL * S * st.P - (w.two ? 1 : 0), flag)) return;
        __nv_bfloat16 *q = st.d + i;
        if (w.two)
            __stcs(reinterpret_cast<__nv_bfloat162 *>(q), __floats2bfloat162_rn(g.x - e.x, g.y - e.y));
        else
            __stcs(q, __float2bfloat16_rn(g.x - e.x));
    }
    __device__ __forceinline__ void put_f(const Site &w, long long plane, float v) const
    {
        const long long i = plane * st.P + w.cell;
        if (in_bounds(i, (long long)(S + 3) * st.P, flag)) __stcs(st.mom + i, v);
    }
    __device__ __forceinline__ void put_f(const Site &w, long long plane, float2 v) const
    {
        const long long i = plane * st.P + w.cell;
        if (!in_bounds(i, (long long)(S + 3) * st.P - (w.two ? 1 : 0), flag)) return;
        float *q = st.mom + i;
        if (w.two)
            __stcs(reinterpret_cast<float2 *>(q), v);
        else
            __stcs(q, v.x);
    }
    template <class V>
    __device__ __forceinline__ void put_n(const Site &w, int s, V n) const
    {
        put_f(w, s, n);
    }
    template <class V>
    __device__ __forceinline__ void put_mix(const Site &w, V ux, V uy, V T) const
    {
        put_f(w, S, ux);
        put_f(w, S + 1, uy);
        put_f(w, S + 2, T);
    }
    __device__ __forceinline__ void images(const Site &, int) const {}
    __device__ __forceinline__ void images_mix(const Site &) const {}
};

// f of species s at one cell (element offset `cell` in a plane), FP32.
template <int S>
__device__ __forceinline__ void bf_cell_f(const StepConsts<float, S> &k, const BfState &st, int s, long long cell,
                                          float f[Q])
{
    const float n = st.mom[(long long)s * st.P + cell];
    const float ux = st.mom[(long long)S * st.P + cell];
    const float uy = st.mom[(long long)(S + 1) * st.P + cell];
    const float T = st.mom[(long long)(S + 2) * st.P + cell];
    feq_ref<S>(k, s, n, ux, uy, T, f);
#pragma unroll
    for (int i = 0; i < Q; ++i) f[i] += __bfloat162float(st.d[(long long)(s * Q + i) * st.P + cell]);
}

// Source policy of the FP64 output kernels for a BF16-deviation state.
template <int S>
struct BfSrc {
    StepConsts<float, S> k;
    BfState st;
    __device__ __forceinline__ void load16(int s, long long cell, double v[Q]) const
    {
        float f[Q];
        bf_cell_f<S>(k, st, s, cell, f);
#pragma unroll
        for (int i = 0; i < Q; ++i) v[i] = (double)f[i];
    }
    __device__ __forceinline__ void load16f(int s, long long cell, float v[Q]) const
    {
        bf_cell_f<S>(k, st, s, cell, v);
    }
};

inline BfState bf_state(const dbm_handle *h, void *buf)
{
    BfState s;
    s.d = (__nv_bfloat16 *)buf;
    s.mom = (float *)((char *)buf + h->lay.moments_offset);
    s.P = h->lay.plane;
    return s;
}

}  // namespace dbm
