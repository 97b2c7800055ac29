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

// ---- node-major full couplings -------------------------------------------
// The refined solver keeps all 27 couplings of every node in 7 groups of
// float4 ([7][N], group g holds offsets t = 4g .. 4g+3; t = 27 is padding
// with coefficient 0): a row is 7 coalesced 16-byte loads at addresses known
// from n alone.  Couplings to nodes outside the mesh are 0, and so is the
// staged value there, so rows need no neighbour checks.
constexpr int kGroups = 7;

__host__ __device__ constexpr int t_dh(int t) {
    return t >= 27 ? 0 : (t % 3 - 1) + SHX * ((t / 3) % 3 - 1) + SHX * SHY * (t / 9 - 1);
}

// FP32 row: sum_t c(t) x(h + dh(t)), t = 0..26 in order
__device__ __forceinline__ float row_f32(const float4* __restrict__ c, size_t N, const float* xs, int h,
                                         int n) {
    float acc = 0.f;
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
        const float4 cv = c[(size_t)g * N + n];
        acc = fmaf(cv.x, xs[h + t_dh(4 * g)], acc);
        acc = fmaf(cv.y, xs[h + t_dh(4 * g + 1)], acc);
        acc = fmaf(cv.z, xs[h + t_dh(4 * g + 2)], acc);
        if (g < kGroups - 1) acc = fmaf(cv.w, xs[h + t_dh(4 * g + 3)], acc);
    }
    return acc;
}

// FP32 row of node n with neighbour values read from global memory
// (node-parallel kernels): sum_t c(t) x(n + off(t)), t = 0..26 in order
__device__ __forceinline__ float row32_np(const float4* __restrict__ c, size_t N, const float* __restrict__ x,
                                          int n, const NbrOff& o) {
    float acc = 0.f;
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
        const float4 cg = c[(size_t)g * N + n];
        const float cv[4] = {cg.x, cg.y, cg.z, cg.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = 4 * g + q;
            if (t < 27) acc = fmaf(cv[q], x[n + o.x[t % 3] + o.y[(t / 3) % 3] + o.z[t / 9]], acc);
        }
    }
    return acc;
}

// float-float row of node n with neighbour values read from global memory
// (node-parallel kernels): (sh + sl) = sum_t (chi + clo)(t) (xh + xl)(n +
// off(t)), t = 0..26 in order, normalised
__device__ __forceinline__ void row_ff_np(const float4* __restrict__ chi, const float4* __restrict__ clo,
                                          size_t N, const float* __restrict__ xh, const float* __restrict__ xl,
                                          int n, const NbrOff& o, float& sh, float& sl) {
    sh = 0.f;
    sl = 0.f;
#pragma unroll
    for (int g = 0; g < kGroups; ++g) {
        const float4 a = chi[(size_t)g * N + n];
        const float4 b = clo[(size_t)g * N + n];
        const float av[4] = {a.x, a.y, a.z, a.w}, bv[4] = {b.x, b.y, b.z, b.w};
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int t = 4 * g + q;
            if (t >= 27) continue;
            const int m = n + o.x[t % 3] + o.y[(t / 3) % 3] + o.z[t / 9];
            ff_mac(av[q], bv[q], xh[m], xl[m], sh, sl);
        }
    }
    ff_normalize(sh, sl);
}

}  // namespace epk
