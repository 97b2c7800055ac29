// ep_tile.cuh -- tiles of the structured meshes for the 27-point stencil
// kernels (shared-memory staging of a vector on a tile plus halo, one stencil
// row from shared memory).
#pragma once

#include "ep_dev.cuh"
#include "ep_ff.cuh"

namespace epk {

// Tiled 27-point applies.  A block loops over tiles of kStTx x kStTy x kStTz
// owned nodes (a persistent grid of about two blocks per SM, one reduction
// per block).  Per tile it stages the input vector on the tile plus a
// one-node halo in shared memory -- forming the CG direction update on the
// way in where the kernel needs it -- together with the global index of
// every halo node (-1 outside the mesh; the periodic direction wraps), then
// each thread applies the stencil to its owned nodes: the 14 own couplings
// are read coalesced, the 13 backward couplings from the neighbours' slots,
// the vector from shared memory.  Summation order is fixed (the diagonal,
// then offsets t = 0..26), so every node rounds the same way in every run.

constexpr int SHX = kStTx + 2, SHY = kStTy + 2, SHZ = kStTz + 2;
constexpr int SHN = SHX * SHY * SHZ;
constexpr int kStOwned = kStTx * kStTy * kStTz;

struct TileGeo {
    int i0, j0, k0;
};

__device__ __forceinline__ TileGeo tile_geo(const Dev& D, int tile) {
    const int tx = (D.NX + kStTx - 1) / kStTx, ty = (D.NY + kStTy - 1) / kStTy;
    TileGeo g;
    g.i0 = (tile % tx) * kStTx;
    g.j0 = ((tile / tx) % ty) * kStTy;
    g.k0 = (tile / (tx * ty)) * kStTz;
    return g;
}

// XF(n, owned) returns the input at node n (and may record it when owned).
template <typename T, class XF>
__device__ __forceinline__ void stage_tile(const Dev& D, const TileGeo& g, int* sidx, T* xs, XF xf) {
    for (int h = threadIdx.x; h < SHN; h += blockDim.x) {
        const int hi = h % SHX, hj = (h / SHX) % SHY, hk = h / (SHX * SHY);
        const int gi = g.i0 - 1 + hi, gk = g.k0 - 1 + hk, gj_raw = g.j0 - 1 + hj;
        bool valid = gi >= 0 && gi < D.NX && gk >= 0 && gk < D.NZ;
        int gj = gj_raw;
        if (D.periodic) gj = ((gj_raw % D.NY) + D.NY) % D.NY;
        else valid = valid && gj_raw >= 0 && gj_raw < D.NY;
        const bool owned = valid && hi >= 1 && hi <= kStTx && hj >= 1 && hj <= kStTy && hk >= 1 &&
                           hk <= kStTz && gj_raw >= 0 && gj_raw < D.NY;
        const int n = valid ? gi + D.NX * (gj + D.NY * gk) : -1;
        sidx[h] = n;
        xs[h] = valid ? xf(n, owned) : T(0);
    }
}

// one stencil row: node n sits at halo position h
template <typename C, typename Acc, typename T>
__device__ __forceinline__ Acc tile_row(const C* __restrict__ c, size_t N, const int* sidx, const T* xs,
                                        int h, int n) {
    Acc acc = (Acc)c[n] * (Acc)xs[h];
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        if (t == 13) continue;
        const int dh = (t % 3 - 1) + SHX * ((t / 3) % 3 - 1) + SHX * SHY * (t / 9 - 1);
        const int m = sidx[h + dh];
        if (m < 0) continue;
        const Acc cv = (t > 13) ? (Acc)c[(size_t)(t - 13) * N + n] : (Acc)c[(size_t)(13 - t) * N + m];
        acc += cv * (Acc)xs[h + dh];
    }
    return acc;
}

// calls f(h, n) for every owned node of the tile this thread handles
template <class F>
__device__ __forceinline__ void for_owned(const Dev& D, const TileGeo& g, F f) {
    for (int o = threadIdx.x; o < kStOwned; o += blockDim.x) {
        const int li = o % kStTx, lj = (o / kStTx) % kStTy, lk = o / (kStTx * kStTy);
        if (g.i0 + li >= D.NX || g.j0 + lj >= D.NY || g.k0 + lk >= D.NZ) continue;
        const int h = (li + 1) + SHX * ((lj + 1) + SHY * (lk + 1));
        f(h);
    }
}

__host__ __device__ inline int st_tiles(const Dev& h) {
    return ((h.NX + kStTx - 1) / kStTx) * ((h.NY + kStTy - 1) / kStTy) * ((h.NZ + kStTz - 1) / kStTz);
}

// index offsets of the 27 neighbours of node n (di, dj, dk in -1..1), from
// its boundary flags; a neighbour outside the mesh maps to a valid node whose
// coupling is 0
struct NbrOff {
    int x[3], y[3], z[3];
};

__device__ __forceinline__ NbrOff nbr_offsets(int nx, int nxy, int wrap, unsigned int f) {
    NbrOff o;
    o.x[0] = (f & 1u) ? 0 : -1;
    o.x[1] = 0;
    o.x[2] = (f & 2u) ? 0 : 1;
    o.y[0] = (f & 4u) ? wrap : -nx;
    o.y[1] = 0;
    o.y[2] = (f & 8u) ? -wrap : nx;
    o.z[0] = (f & 16u) ? 0 : -nxy;
    o.z[1] = 0;
    o.z[2] = (f & 32u) ? 0 : nxy;
    return o;
}

// ---- symmetric float stencils -------------------------------------------
// The refined solver keeps A (and, on curved meshes, M) as float-float pairs
// in the slots of the FP64 stencils: per node the diagonal (slot 0) and the
// 13 forward couplings (slot s = 1..13, offset t = 13 + s), slot s of node n
// at s * cs + n.  The coupling of node n to its backward neighbour
// m = n + off(t), t < 13, is m's forward slot 13 - t: the operators are
// symmetric, so a row reads 14 values at n and 13 at its backward
// neighbours instead of 27 stored per node (half the bytes).  Couplings to
// forward neighbours outside the mesh are stored as 0.  A backward neighbour
// outside the mesh is either masked by the node's boundary flags or -- on a
// slab read at fixed offsets -- lands on a node whose coupling in the
// reverse direction leaves the mesh (so is 0) or in the zero padding before
// the arrays.  Rows sum t = 0..26 in order, so they round exactly as rows of
// the 27 couplings stored per node would.

__host__ __device__ constexpr int t_dh(int t) {
    return t >= 27 ? 0 : (t % 3 - 1) + SHX * ((t / 3) % 3 - 1) + SHX * SHY * (t / 9 - 1);
}

// boundary-flag bits (i = 0, i = NX-1, j = 0, j = NY-1, k = 0, k = NZ-1) that
// put the neighbour at offset t outside the mesh
__host__ __device__ constexpr unsigned int off_bits(int t) {
    return ((t % 3 == 0) ? 1u : 0u) | ((t % 3 == 2) ? 2u : 0u) | (((t / 3) % 3 == 0) ? 4u : 0u) |
           (((t / 3) % 3 == 2) ? 8u : 0u) | ((t / 9 == 0) ? 16u : 0u) | ((t / 9 == 2) ? 32u : 0u);
}

// the flags that matter for neighbour existence: j wraps on periodic meshes
__device__ __forceinline__ unsigned int exist_flags(unsigned int f, int wrap) { return wrap ? (f & ~12u) : f; }

// coupling of node n at offset t (neighbour m); MASK: zero it when the
// flags fe put the neighbour outside the mesh
template <bool MASK>
__device__ __forceinline__ float sym_coupling(const float* __restrict__ A, long long cs, int n, int m, int t,
                                              unsigned int fe) {
    if (t == 13) return A[n];
    if (t > 13) return A[(long long)(t - 13) * cs + n];
    const float c = A[(long long)(13 - t) * cs + m];
    return (MASK && (fe & off_bits(t))) ? 0.f : c;
}

// ---- L2 eviction-priority hints -------------------------------------------
// An access policy (createpolicy) attached to loads and stores: lines fetched
// under evict_last are kept in L2 in preference to others, evict_first lines
// are dropped first.  The persistent solve streams the operator's couplings
// (read once per pass) under evict_first and keeps its CG vectors under
// evict_last, so that the vectors of an instance whose whole working set
// exceeds L2 stay resident across passes.
__device__ __forceinline__ unsigned long long l2_policy_evict_last() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_last.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ unsigned long long l2_policy_evict_first() {
    unsigned long long p;
    asm volatile("createpolicy.fractional.L2::evict_first.b64 %0, 1.0;" : "=l"(p));
    return p;
}

__device__ __forceinline__ float ld_pol(const float* a, unsigned long long pol) {
    float v;
    asm("ld.global.L2::cache_hint.f32 %0, [%1], %2;" : "=f"(v) : "l"(a), "l"(pol));
    return v;
}

__device__ __forceinline__ void st_pol(float* a, float v, unsigned long long pol) {
    asm volatile("st.global.L2::cache_hint.f32 [%0], %1, %2;" ::"l"(a), "f"(v), "l"(pol) : "memory");
}

// FP32 row of node n as row32_sym, couplings read under policy pa and the
// vector under pv
__device__ __forceinline__ float row32_sym_pol(const float* __restrict__ A, long long cs,
                                               const float* __restrict__ x, int n, const NbrOff& o,
                                               unsigned int fe, unsigned long long pa, unsigned long long pv) {
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        const int m = n + o.x[t % 3] + o.y[(t / 3) % 3] + o.z[t / 9];
        float c;
        if (t == 13) c = ld_pol(A + n, pa);
        else if (t > 13) c = ld_pol(A + (long long)(t - 13) * cs + n, pa);
        else c = (fe & off_bits(t)) ? 0.f : ld_pol(A + (long long)(13 - t) * cs + m, pa);
        acc = fmaf(c, ld_pol(x + m, pv), acc);
    }
    return acc;
}

// FP32 row with neighbour values staged in shared memory (tiled kernels):
// sum_t c(t) x(h + dh(t)), t = 0..26 in order; sidx[h'] is the node index
// at halo position h' (-1 outside the mesh)
__device__ __forceinline__ float row_f32_sym(const float* __restrict__ A, long long cs, const int* sidx,
                                             const float* xs, int h, int n) {
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        float c;
        if (t >= 13) {
            c = sym_coupling<false>(A, cs, n, n, t, 0u);
        } else {
            const int m = sidx[h + t_dh(t)];
            c = m < 0 ? 0.f : A[(long long)(13 - t) * cs + m];
        }
        acc = fmaf(c, xs[h + t_dh(t)], acc);
    }
    return acc;
}

// FP32 row of node n with neighbour values read from global memory
// (node-parallel kernels): sum_t c(t) x(n + off(t)), t = 0..26 in order
template <bool MASK>
__device__ __forceinline__ float row32_sym(const float* __restrict__ A, long long cs,
                                           const float* __restrict__ x, int n, const NbrOff& o,
                                           unsigned int fe) {
    float acc = 0.f;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        const int m = n + o.x[t % 3] + o.y[(t / 3) % 3] + o.z[t / 9];
        acc = fmaf(sym_coupling<MASK>(A, cs, n, m, t, fe), x[m], acc);
    }
    return acc;
}

// float-float row of node n with neighbour values read from global memory
// (node-parallel kernels, boundary flags fe): (sh + sl) = sum_t (chi + clo)(t)
// (xh + xl)(n + off(t)), t = 0..26 in order, normalised
__device__ __forceinline__ void row_ff_sym(const float* __restrict__ chi, const float* __restrict__ clo,
                                           long long cs, const float* __restrict__ xh,
                                           const float* __restrict__ xl, int n, const NbrOff& o,
                                           unsigned int fe, float& sh, float& sl) {
    sh = 0.f;
    sl = 0.f;
#pragma unroll
    for (int t = 0; t < 27; ++t) {
        const int m = n + o.x[t % 3] + o.y[(t / 3) % 3] + o.z[t / 9];
        const float ch = sym_coupling<true>(chi, cs, n, m, t, fe);
        const float cl = sym_coupling<true>(clo, cs, n, m, t, fe);
        ff_mac(ch, cl, xh[m], xl[m], sh, sl);
    }
    ff_normalize(sh, sl);
}

}  // namespace epk
