// k_pcg.cu -- the whole linear solve of a step, every refinement sweep, in
// one persistent, cooperative launch (stencil operator): the FP32 inner solve,
// the correction and the float-float residual with the refinement's decision.
//
// Jacobi-preconditioned CG (the paper solves Eq. (6) with CG, Sec. 2) on
// A delta = r in float, A the hi parts of the symmetric float-float stencil, in
// the single-reduction arrangement of Chronopoulos and Gear (1989): with
// u = D^-1 r and w = A u, both dot products of an iteration come from the
// same pass.  Iteration i, given alpha_i and beta_i:
//   update (every node on its own):
//     s_i = w_i + beta_i s_{i-1},   r_{i+1} = r_i - alpha_i s_i,
//     p_i = u_i + beta_i p_{i-1},   delta  += alpha_i p_i,   u_{i+1} = D^-1 r_{i+1}
//   grid barrier (u_{i+1} of the neighbours is needed next)
//   apply: w_{i+1} = A u_{i+1}; block partials of
//     gamma = (r_{i+1}, u_{i+1}), eta = (u_{i+1}, w_{i+1}), rho = (r_{i+1}, r_{i+1})
//   grid barrier; every block sums all partials in the same fixed order, so
//   all blocks take the same
//     beta_{i+1} = gamma_{i+1} / gamma_i,
//     alpha_{i+1} = gamma_{i+1} / (eta_{i+1} - beta_{i+1} gamma_{i+1} / alpha_i)
//   and the same stopping decision (rho relative to the sweep's first rho).
// The right-hand-side kernel leaves r_0 and u_0 = D^-1 r_0, so the launch
// starts with the apply of u_0.  Nodes are spread over all threads of the
// grid in index order (thread t: nodes t, t + T, ...), so every thread owns
// the same number of nodes up to one.  Neighbour values of u are plain
// cached loads: they were written before the last barrier, whose
// release/acquire pair orders them for every thread of the block; on a Q1
// slab u is padded with zeros, so rows read their neighbours at fixed
// offsets without the boundary flags.  A barrier that does not complete
// within ~1 s records EP_ETIMEOUT and the kernel returns.
//
// A pipelined arrangement (Ghysels and Vanroose 2014: w and z = A D^-1 s by
// recurrence, one pass and one barrier per iteration) measured the same on
// the 442k-node slab (331 against 333 us a step's solve) and slower on the
// LV shell, where the float recurrences slowed convergence (100 inner
// iterations a sweep against 36); it is not used.
//
// After the inner solve: u += delta (float-float), a grid barrier, then the
// residual of the sweep on the same node map -- y = A u with the float-float
// couplings, r = b - y, the next inner solve's start (r, D^-1 r, delta = 0) --
// and its sums (ns b)^2, (ns r)^2, r . D^-1 r, r . r, reduced like the CG's
// (block partials, every block summing them in the same order), so every
// block takes the same decision: the refinement has converged when
// ||r|| <= tol ||b||, else another sweep follows (at most max_sweeps); block 0
// records the step's figures and, at the end, rotates the time levels.  The
// inner solve's couplings are then still in L2 for the residual's hi parts.
#include "ep_dev.cuh"
#include "ep_ff.cuh"
#include "ep_tile.cuh"

namespace epk {

constexpr long long kBarrierSpinLimit = 1ll << 24;  // x >= 64 ns naps: about a second

// Bounded grid barrier (all blocks of a cooperative launch) on a 64-bit
// arrival counter that only grows: every barrier adds exactly one arrival
// per block, so barrier k of a launch completes when the counter reaches
// base + k G, base being the counter at launch start (a multiple of G).
// Thread 0 of each block arrives with one acq_rel atomic and waits with
// acquire loads; the block's other threads are ordered behind it by
// __syncthreads.  `target` is thread 0's running target (0 before the first
// barrier of the launch).  Returns false after recording EP_ETIMEOUT when the
// other blocks did not all arrive in time.  (A release reduction for the
// arrival with relaxed polling and one acquire fence measured slower: 1930
// against 1910 us a step's solve on the 2.19M-node shell, 354 against 339 us
// on the 442k-node slab.)
__device__ __forceinline__ bool grid_barrier(unsigned long long* count, unsigned long long& target, int G,
                                             int* status, long long spin_limit = kBarrierSpinLimit) {
    __shared__ int ok;
    __syncthreads();
    if (threadIdx.x == 0) {
        int good = 1;
        unsigned long long old;
        asm volatile("atom.add.acq_rel.gpu.u64 %0, [%1], 1;" : "=l"(old) : "l"(count) : "memory");
        const unsigned long long g = (unsigned long long)G;
        target = (target == 0ull ? old - old % g : target) + g;
        long long spins = 0;
        for (;;) {
            unsigned long long cur;
            asm volatile("ld.acquire.gpu.u64 %0, [%1];" : "=l"(cur) : "l"(count) : "memory");
            if (cur >= target) break;
            if (++spins > spin_limit) {
                good = 0;
                atomicCAS(status, (int)EP_OK, (int)EP_ETIMEOUT);
                break;
            }
            __nanosleep(20);
        }
        ok = good;
    }
    __syncthreads();
    return ok != 0;
}

// ---- tiled apply ------------------------------------------------------------
// On structured Q1 meshes whose solve does not fit in L2, the apply pass can
// run on tiles instead of the node-parallel map: block b owns the nodes of
// tile_by consecutive rows j (every i) over a contiguous range of k planes
// and walks its planes in order.  The bulk-copy (TMA) unit stages each plane
// of the tile in shared memory -- the tile's rows with one row of halo on
// either side and one float of slack at either end, which in the compact node
// order is one contiguous range, so one bulk copy per slot (16-byte aligned:
// the range widened to multiples of four floats and indexed from the
// remainder).  The 14 coupling slots of plane k + 1 and u of plane k + 2 are
// in flight while plane k is applied (three coupling and four u buffers in a
// ring, one mbarrier each), so the operator's DRAM stream runs
// asynchronously, and every row reads its 27 couplings and 27 neighbour
// values from shared memory at fixed offsets: the node at q = (j - j0) NX + i
// of the tile has its neighbour (di, dj) at q + (dj + 1) NX + (di + 1) from the
// plane's first copied node.
//
// The halo rows are the compact order's neighbours: past the i boundary the
// adjacent row's last or first node, past the mesh's j or k boundary the
// next plane's row or the zero padding around the arrays -- all of them
// nodes whose coupling towards the tile's node is zero (as for the padded
// slab's fixed offsets).  A periodic mesh's seam rows (j = -1 is row NY - 1,
// j = NY is row 0) are patched over the halo row once the plane has landed,
// from 4-byte asynchronous copies issued a plane ahead into a staging area.
// Planes outside the mesh are buffers of zeros.  Each row sums t = 0..26 in
// the node-parallel order; only the dot products' partials are grouped by
// tile.
//
// Measured on the 2.19M-node LV shell (tiles of 50 rows over 13-14 planes,
// 152 blocks): 2.43 ms a step's solve against 1.85 ms for the node-parallel
// apply.  Three coupling planes of 62 KB fill the shared memory, so a block
// has about one plane of copies in flight, while the node-parallel apply
// keeps each thread's 27 coupling loads in flight (32 warps an SM): the
// copies wait on DRAM latency and the pass runs at about half the
// bandwidth.  An L2 prefetch of the planes three ahead (bulk prefetches)
// made it slower still (2.95 ms), and so did tiles of 48 rows (one node per
// thread and plane).  The tiled apply is kept as an option
// (ep_options.solve_tiles = 2).

constexpr long long kStageWaitLimit = 1ll << 22;  // try_wait rounds (each suspends for a while)

__device__ __forceinline__ unsigned int sm_addr(const void* p) {
    return (unsigned int)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_expect(unsigned int bar, unsigned int bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}

template <bool HINT>
__device__ __forceinline__ void bulk_g2s(unsigned int dst, const float* src, unsigned int bytes, unsigned int bar,
                                         unsigned long long pol) {
    if (HINT)
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes.L2::cache_hint"
            " [%0], [%1], %2, [%3], %4;" ::"r"(dst),
            "l"(src), "r"(bytes), "r"(bar), "l"(pol)
            : "memory");
    else
        asm volatile(
            "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];" ::"r"(dst),
            "l"(src), "r"(bytes), "r"(bar)
            : "memory");
}

// Bounded wait for the phase of the given parity; false when it did not
// complete within the limit.
__device__ __forceinline__ bool mbar_wait(unsigned int bar, unsigned int parity) {
    for (long long i = 0; i < kStageWaitLimit; ++i) {
        unsigned int done;
        asm volatile(
            "{\n\t.reg .pred p;\n\t"
            "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
            "selp.u32 %0, 1, 0, p;\n\t}"
            : "=r"(done)
            : "r"(bar), "r"(parity)
            : "memory");
        if (done) return true;
    }
    return false;
}

// A block's tile (block-uniform).
struct TileBlk {
    int j0, rows, k0, k1;
    bool seam_lo, seam_hi;   // periodic: row j0 - 1 = -1 is row NY - 1; row j0 + rows = NY is row 0
    int L;                   // floats per slot and plane
};

__device__ __forceinline__ TileBlk tile_of(const Dev& D, int blk) {
    TileBlk T;
    const int jt = blk / D.tile_kr, kr = blk - jt * D.tile_kr;
    T.j0 = jt * D.tile_by;
    T.rows = min(D.tile_by, D.NY - T.j0);
    T.k0 = (int)((long long)kr * D.NZ / D.tile_kr);
    T.k1 = (int)((long long)(kr + 1) * D.NZ / D.tile_kr);
    T.seam_lo = D.periodic && T.j0 == 0;
    T.seam_hi = D.periodic && T.j0 + T.rows == D.NY;
    T.L = D.tile_l;
    return T;
}

// Node index of plane kk's first copied node (the slack before row j0 - 1),
// and the first float of its copy (rounded down to 16 bytes): the plane's
// nodes sit (first - copy start) floats into its buffer.
__device__ __forceinline__ long long tile_first(const TileBlk& T, int NX, int NXY, int kk) {
    return (long long)kk * NXY + (long long)(T.j0 - 1) * NX - 1;
}

__device__ __forceinline__ int tile_shift(const TileBlk& T, int NX, int NXY, int kk) {
    return (int)(tile_first(T, NX, NXY, kk) & 3ll);
}

// Thread 0: the bulk copy of plane kk of nslot slots of src (slot stride cs)
// into the plane buffer dst (slot stride L), completing on bar.
template <bool HINT>
__device__ __forceinline__ void stage_plane(const TileBlk& T, int NX, int NXY, const float* src, long long cs,
                                            int nslot, float* dst, unsigned int bar, int kk,
                                            unsigned long long pol) {
    const long long g0 = tile_first(T, NX, NXY, kk);
    const long long m0 = g0 & ~3ll;
    const long long m1 = (g0 + (long long)(T.rows + 2) * NX + 2 + 3) & ~3ll;
    const unsigned int bm = (unsigned int)((m1 - m0) * 4);
    mbar_expect(bar, (unsigned int)nslot * bm);
    for (int sl = 0; sl < nslot; ++sl)
        bulk_g2s<HINT>(sm_addr(dst + (size_t)sl * T.L), src + (long long)sl * cs + m0, bm, bar, pol);
}

// The seam rows of a periodic tile: NX + 1 floats per slot and seam, the
// lower one (row NY - 1 from the node before it, as row -1) at positions
// 0 .. NX, the upper one (row 0 and the node after it, as row NY) at
// (rows + 1) NX + 1 ... of a plane.  Element x of a plane's seam floats:
// the seam (lower first), the slot, the position; its source node index
// (slot offset apart) and its position from the plane's first node.
__device__ __forceinline__ void seam_elem(const TileBlk& T, int NX, int NY, int NXY, int nslot, int kk, int x,
                                          int& slot, long long& src, int& pos) {
    const int per = nslot * (NX + 1);
    const bool hi = !T.seam_lo || x >= per;
    const int rem = x >= per ? x - per : x;
    slot = rem / (NX + 1);
    const int e = rem - slot * (NX + 1);
    const long long pb = (long long)kk * NXY;
    if (hi) {
        src = pb + e;
        pos = (T.rows + 1) * NX + 1 + e;
    } else {
        src = pb + (long long)(NY - 1) * NX - 1 + e;
        pos = e;
    }
}

__device__ __forceinline__ int seam_count(const TileBlk& T, int NX, int nslot) {
    return ((T.seam_lo ? 1 : 0) + (T.seam_hi ? 1 : 0)) * nslot * (NX + 1);
}

// Dynamic shared memory of the tiled apply for l floats per slot and plane:
// 128 bytes of mbarriers, three coupling planes of 14 slots, four planes of
// u, and the seam rows' staging (two seams of 15 slots).
size_t tiled_smem_bytes(int l, int NX) {
    return 128 + (size_t)(3 * kSlots + 4) * (size_t)l * sizeof(float) +
           (size_t)2 * (kSlots + 1) * (NX + 1) * sizeof(float);
}

// All threads: zeros over n floats at p (a plane outside the mesh).
__device__ __forceinline__ void zero_floats(float* p, int n) {
    for (int x = threadIdx.x; x < n; x += blockDim.x) p[x] = 0.f;
}

// The apply pass on the block's tile: w = A u on its nodes and the partials
// gamma = (r, u), eta = (u, w), rho = (r, r).  cpar / upar: the parity bits
// of the coupling / u buffers' mbarriers (block-uniform).  Every copy issued
// here is waited for here.  Returns false (after recording EP_ETIMEOUT and
// waiting, bounded, for the copies in flight) when a copy did not complete.
template <int BT, bool HINT>
__device__ __forceinline__ bool apply_tiled(Dev& D, const TileBlk& T, unsigned int& cpar, unsigned int& upar,
                                            const float* __restrict__ u, const float* __restrict__ r,
                                            float* __restrict__ w, float (&v)[3], unsigned long long pkeep,
                                            unsigned long long pstream) {
    extern __shared__ __align__(128) float dsm[];
    const int NX = D.NX, NY = D.NY, NZ = D.NZ, NXY = D.NX * D.NY;
    const long long cs = D.cs;
    const float* A = D.Ahi;
    const int L = T.L;
    const unsigned int bar0 = sm_addr(dsm);  // 7 mbarriers: couplings 0..2, u 3..6
    float* CB = dsm + 32;
    float* UB = CB + (size_t)3 * kSlots * L;
    float* SC = UB + (size_t)4 * L;          // staging of the seam rows: couplings
    float* SU = SC + 2 * kSlots * (NX + 1);  // and u
    const int nsc = seam_count(T, NX, kSlots), nsu = seam_count(T, NX, 1);
    unsigned int cout = 0u, uout = 0u;  // buffers in flight
    auto cbuf = [&](int kk) { return (kk + 3) % 3; };
    auto ubuf = [&](int kk) { return (kk + 4) % 4; };
    // a plane's first copied node in its buffer
    auto cplane = [&](int kk) {
        return CB + (size_t)cbuf(kk) * kSlots * L + tile_shift(T, NX, NXY, kk);
    };
    auto uplane = [&](int kk) { return UB + (size_t)ubuf(kk) * L + tile_shift(T, NX, NXY, kk); };
    auto inside = [&](int kk) { return kk >= 0 && kk < NZ; };
    // a plane in the mesh is copied (thread 0 issues, every thread records it
    // in flight); one outside is filled with zeros by all threads
    auto stage_c = [&](int kk) {
        const int b = cbuf(kk);
        if (!inside(kk)) {
            zero_floats(CB + (size_t)b * kSlots * L, kSlots * L);
            return;
        }
        if (threadIdx.x == 0)
            stage_plane<HINT>(T, NX, NXY, A, cs, kSlots, CB + (size_t)b * kSlots * L, bar0 + 8u * b, kk, pstream);
        cout |= 1u << b;
    };
    auto stage_u = [&](int kk) {
        const int b = ubuf(kk);
        if (!inside(kk)) {
            zero_floats(UB + (size_t)b * L, L);
            return;
        }
        if (threadIdx.x == 0)
            stage_plane<HINT>(T, NX, NXY, u, 0, 1, UB + (size_t)b * L, bar0 + 8u * (3 + b), kk, pkeep);
        uout |= 1u << b;
    };
    bool ok = true;
    // (a wait that gives up leaves its buffer in flight, for the drain below)
    auto wait_c = [&](int kk) {
        const int b = cbuf(kk);
        if (!((cout >> b) & 1u)) return;
        if (mbar_wait(bar0 + 8u * b, (cpar >> b) & 1u)) {
            cpar ^= 1u << b;
            cout &= ~(1u << b);
        } else {
            ok = false;
        }
    };
    auto wait_u = [&](int kk) {
        const int b = ubuf(kk);
        if (!((uout >> b) & 1u)) return;
        if (mbar_wait(bar0 + 8u * (3 + b), (upar >> b) & 1u)) {
            upar ^= 1u << b;
            uout &= ~(1u << b);
        } else {
            ok = false;
        }
    };
    // seam rows of plane kk (periodic tiles at the seam): loaded directly,
    // or copied into the staging area (4-byte asynchronous copies) and
    // patched in from there once the plane has landed
    auto seam_direct = [&](int kk, bool coup) {
        if (!inside(kk)) return;
        const int n = coup ? nsc : nsu;
        float* base = coup ? cplane(kk) : uplane(kk);
        for (int x = threadIdx.x; x < n; x += BT) {
            int sl, pos;
            long long g;
            seam_elem(T, NX, NY, NXY, coup ? kSlots : 1, kk, x, sl, g, pos);
            base[(size_t)sl * L + pos] = coup ? A[(long long)sl * cs + g] : u[g];
        }
    };
    auto seam_issue = [&](int kk, bool coup) {
        if (!inside(kk)) return;
        const int n = coup ? nsc : nsu;
        float* st = coup ? SC : SU;
        for (int x = threadIdx.x; x < n; x += BT) {
            int sl, pos;
            long long g;
            seam_elem(T, NX, NY, NXY, coup ? kSlots : 1, kk, x, sl, g, pos);
            const float* a = coup ? A + (long long)sl * cs + g : u + g;
            asm volatile("cp.async.ca.shared.global [%0], [%1], 4;" ::"r"(sm_addr(st + x)), "l"(a) : "memory");
        }
    };
    auto seam_patch = [&](int kk, bool coup) {
        if (!inside(kk)) return;
        const int n = coup ? nsc : nsu;
        const float* st = coup ? SC : SU;
        float* base = coup ? cplane(kk) : uplane(kk);
        for (int x = threadIdx.x; x < n; x += BT) {
            int sl, pos;
            long long g;
            seam_elem(T, NX, NY, NXY, coup ? kSlots : 1, kk, x, sl, g, pos);
            base[(size_t)sl * L + pos] = st[x];
        }
    };
    const bool seams = nsc > 0;
    const int k0 = T.k0, k1 = T.k1;
    if (threadIdx.x == 0) {
        // u was written by other blocks before the grid barrier (generic
        // proxy); the bulk copies read it through the async proxy
        asm volatile("fence.proxy.async.global;" ::: "memory");
        asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    }
    stage_c(k0 - 1);
    stage_c(k0);
    stage_u(k0 - 1);
    stage_u(k0);
    stage_u(k0 + 1);
    wait_c(k0 - 1);
    wait_c(k0);
    wait_u(k0 - 1);
    wait_u(k0);
    wait_u(k0 + 1);
    if (seams) {
        seam_direct(k0 - 1, true);
        seam_direct(k0, true);
        seam_direct(k0 - 1, false);
        seam_direct(k0, false);
        seam_direct(k0 + 1, false);
    }
    float v0 = 0.f, v1 = 0.f, v2 = 0.f;
    bool bad = false;
    for (int k = k0; k < k1 && !bad; ++k) {
        // the next plane's couplings and the plane after it of u (their
        // buffers were last read for plane k - 1, before the barrier that
        // ended it)
        if (threadIdx.x == 0) asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
        if (k + 1 < k1) stage_c(k + 1);
        if (k + 2 <= k1) stage_u(k + 2);
        wait_c(k);
        wait_u(k + 1);
        if (seams && k > k0) {
            // the seam rows staged during plane k - 1
            asm volatile("cp.async.wait_all;" ::: "memory");
            seam_patch(k, true);
            seam_patch(k + 1, false);
        }
        __syncthreads();  // plane k, its seam rows and zero planes in place
        if (seams) {
            if (k + 1 < k1) seam_issue(k + 1, true);
            if (k + 2 <= k1) seam_issue(k + 2, false);
            asm volatile("cp.async.commit_group;" ::: "memory");
        }
        // the rows of plane k: node q of the tile at q + NX + 1 from a
        // plane's first copied node, its neighbour (dx, dy) - 1 at
        // q + dy NX + dx
        const float* cm = cplane(k - 1);
        const float* ck = cplane(k);
        const float* um = uplane(k - 1);
        const float* uk = uplane(k);
        const float* up = uplane(k + 1);
        const int nb = k * NXY + T.j0 * NX;
        const int own_n = T.rows * NX;
        for (int q = threadIdx.x; q < own_n; q += BT) {
            const int n = nb + q;
            const float rn = HINT ? ld_pol(r + n, pkeep) : r[n];
            float acc = 0.f;
#pragma unroll
            for (int t = 0; t < 27; ++t) {
                const int dx = t % 3, dy = (t / 3) % 3, dz = t / 9;
                const int off = q + dy * NX + dx;
                // the diagonal and forward couplings: the node's own slots in
                // plane k; backward: the neighbour's (planes k - 1 and k)
                const float c = t >= 13 ? ck[(t - 13) * L + q + NX + 1] : (dz == 0 ? cm : ck)[(13 - t) * L + off];
                const float* ub = dz == 0 ? um : (dz == 1 ? uk : up);
                acc = fmaf(c, ub[off], acc);
            }
            if (HINT) st_pol(w + n, acc, pkeep);
            else w[n] = acc;
            const float un = uk[q + NX + 1];
            v0 = fmaf(rn, un, v0);
            v1 = fmaf(un, acc, v1);
            v2 = fmaf(rn, rn, v2);
        }
        // every thread is done with plane k - 1's buffers before they are
        // refilled; a copy that did not complete ends the pass everywhere
        bad = __syncthreads_or(!ok) != 0;
    }
    if (seams) asm volatile("cp.async.wait_all;" ::: "memory");  // (none left in flight: see the loop's end)
    v[0] = v0;
    v[1] = v1;
    v[2] = v2;
    if (!bad) return true;
    if (threadIdx.x == 0) atomicCAS(&D.status, (int)EP_OK, (int)EP_ETIMEOUT);
    // the copies still in flight land before the block may leave
    for (int b = 0; b < 3; ++b)
        if ((cout >> b) & 1u) (void)mbar_wait(bar0 + 8u * b, (cpar >> b) & 1u);
    for (int b = 0; b < 4; ++b)
        if ((uout >> b) & 1u) (void)mbar_wait(bar0 + 8u * (3 + b), (upar >> b) & 1u);
    __syncthreads();
    return false;
}

// u += delta (float-float) on this thread's nodes; kept out of line so that
// its registers do not add to the solver loop's
__device__ __noinline__ void correct_ff_nodes(const Dev& D, int t0, int T) {
    float* __restrict__ uh = D.u_hi;
    float* __restrict__ ul = D.u_lo;
    const float* __restrict__ x = D.d32;
    for (int n = t0; n < D.N; n += T) {
        float h = uh[n], l = ul[n];
        ff_add_f(h, l, x[n], h, l);
        uh[n] = h;
        ul[n] = l;
    }
}

// The sweep's float-float residual on this thread's nodes: y = A u with
// the hi and lo couplings (stored as the step's A u), r = b - y, the next
// inner solve's start (r32 = r, z32 = D^-1 r32, delta = 0), and this
// thread's sums (ns b)^2, (ns r)^2, r32 . z32, r32 . r32.  Out of line, as
// correct_ff_nodes.
__device__ __noinline__ void resid_ff_nodes(const Dev& D, int t0, int T, float (&vf)[4]) {
    const int N = D.N;
    const int nx = D.NX, nxy = D.NX * D.NY, wrap = D.periodic ? D.NX * (D.NY - 1) : 0;
    const float ns = D.nscale;
    const float* __restrict__ uh = D.u_hi;
    const float* __restrict__ ul = D.u_lo;
    vf[0] = vf[1] = vf[2] = vf[3] = 0.f;
    const unsigned char* __restrict__ flag = D.nflag;
    unsigned int fn = t0 < N ? flag[t0] : 0u;
    for (int n = t0; n < N; n += T) {
        const unsigned int f = fn;
        fn = n + T < N ? flag[n + T] : 0u;
        const NbrOff o = nbr_offsets(nx, nxy, wrap, f);
        float ah, al, rh, rl;
        row_ff_sym(D.Ahi, D.Alo, D.cs, uh, ul, n, o, exist_flags(f, wrap), ah, al);
        D.yc_hi[n] = ah;
        D.yc_lo[n] = al;
        const float bh = D.b_hi[n];
        ff_sub(bh, D.b_lo[n], ah, al, rh, rl);
        const float r32 = rh;
        const float z = D.dinv32[n] * r32;
        D.r32[n] = r32;
        D.z32[n] = z;
        D.d32[n] = 0.0f;
        const float bs = ns * bh, rs = ns * rh;
        vf[0] = fmaf(bs, bs, vf[0]);
        vf[1] = fmaf(rs, rs, vf[1]);
        vf[2] = fmaf(r32, z, vf[2]);
        vf[3] = fmaf(r32, r32, vf[3]);
    }
}

// BT threads per block, MINB resident blocks per SM; TILED: the apply pass on
// tiles (apply_tiled; one instance, dynamic shared memory).  An instance alone runs
// one 1024-thread block per SM (64 registers, 32 warps in flight, 152
// arrivals at each grid barrier); measured against one 512-thread block
// (128 registers, 16 warps) and two of them (64 registers, 304 arrivals) a
// step's solve took 249.5 / 255.0 / 277.3 us on the 442k-node slab and
// 2086 / 2373 / 2108 us on the 2.19M-node LV shell.  Batches run the same
// 1024-thread blocks, shared among their instances by size (so an instance
// rounds alike alone and in a batch, to its share of blocks).
template <int BT, int MINB, bool HINT, bool TILED>
__global__ void __launch_bounds__(BT, MINB) k_solve32_stencil(Batch B) {
    const Slot S = batch_slot(B);
    Dev& D = *S.D;
    // the step's first residual may already meet the tolerance; a batched
    // launch also visits such instances
    if (!D.f_outer) return;
    const int N = D.N;
    const int G = S.nblk;
    const int T = G * blockDim.x;
    const int t0 = S.blk * blockDim.x + threadIdx.x;
    // mesh sizes in registers for the neighbour offsets
    const int nx = D.NX, nxy = D.NX * D.NY, wrap = D.periodic ? D.NX * (D.NY - 1) : 0;
    float* __restrict__ r = D.r32;
    float* __restrict__ w = D.q32;
    float* __restrict__ s = D.pa32;
    float* __restrict__ p = D.pb32;
    float* __restrict__ x = D.d32;
    const float* __restrict__ dinv = D.dinv32;
    const unsigned char* __restrict__ flag = D.nflag;
    // Q1 slab: u is padded, so every row reads its 27 neighbours at fixed
    // offsets (couplings past the slab's edge are 0) and the boundary flags
    // are not needed
    const bool fixed = D.npad > 0 && wrap == 0;
    const float* __restrict__ A = D.Ahi;
    const long long cs = D.cs;
    // HINT (working set beyond L2): the CG vectors kept in L2, the couplings
    // streamed; otherwise plain accesses (an L2-resident instance gains
    // nothing and its couplings would be dropped first)
    const unsigned long long pkeep = HINT ? l2_policy_evict_last() : 0ull;
    const unsigned long long pstream = HINT ? l2_policy_evict_first() : 0ull;
    auto ldv = [&](const float* a) { return HINT ? ld_pol(a, pkeep) : *a; };
    auto stv = [&](float* a, float v) {
        if (HINT) st_pol(a, v, pkeep);
        else *a = v;
    };
    float* part = reinterpret_cast<float*>(D.partial);
    unsigned long long* bcount = reinterpret_cast<unsigned long long*>(D.counter + CNT_BAR);
    unsigned long long target = 0ull;
    // CG scalars (float, like the solve): formed by thread 0 of every block
    // from the same totals, handed to the block through shared memory
    __shared__ float sc_alpha, sc_beta;
    __shared__ int sc_done, sc_it, sc_nan, sc_more, sc_sweeps, sc_itsum;
    __shared__ float sc_stop, sc_gam_old, sc_alpha_old, sc_rr, sc_gam;
    if (threadIdx.x == 0) {
        sc_it = 0;
        sc_nan = 0;
        sc_sweeps = 0;
        sc_itsum = 0;
        sc_stop = (float)D.inner_stop;  // the first sweep's, from the right-hand side
        sc_gam_old = sc_alpha_old = sc_rr = sc_gam = 0.f;
    }
    // tiled apply: the block's tile and the staging buffers' mbarriers (one
    // arrival per phase, from the thread issuing the copies)
    TileBlk tb{};
    unsigned int cpar = 0u, upar = 0u;
    if constexpr (TILED) {
        tb = tile_of(D, S.blk);
        if (threadIdx.x == 0) {
            extern __shared__ __align__(128) float dsm[];
            const unsigned int bar0 = sm_addr(dsm);
            for (int b = 0; b < 7; ++b) asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(bar0 + 8u * b) : "memory");
            asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
        }
    }
    __syncthreads();
    bool aborted = false;
    for (;;) {  // ---- refinement sweeps
        float alpha = 0.f, beta = 0.f;
        bool first = true;
        if (threadIdx.x == 0) sc_it = 0;
        float* __restrict__ u = D.z32;
        for (;;) {  // ---- inner CG: an update pass and an apply pass per iteration
            if (!first) {
                // ---- update, node by node (L2-bandwidth bound on the
                // 2.19M-node shell: 16-byte accesses, four nodes a thread,
                // measured slower -- 2123 against 1910 us a step's solve)
                for (int n = t0; n < N; n += T) {
                    const float dv = ldv(dinv + n);
                    const float r0 = ldv(r + n), w0 = ldv(w + n), u0 = ldv(u + n);
                    const float s1 = beta == 0.f ? w0 : fmaf(beta, ldv(s + n), w0);
                    const float p1 = beta == 0.f ? u0 : fmaf(beta, ldv(p + n), u0);
                    const float r1 = fmaf(-alpha, s1, r0);
                    stv(x + n, fmaf(alpha, p1, ldv(x + n)));
                    stv(s + n, s1);
                    stv(p + n, p1);
                    stv(r + n, r1);
                    stv(u + n, dv * r1);
                }
                if (!grid_barrier(bcount, target, G, &D.status)) {
                    aborted = true;
                    break;
                }
            }
            // ---- apply w = A u and the block partials
            float v[3] = {0.f, 0.f, 0.f};  // gamma, eta, rho
            if constexpr (TILED) {
                if (!apply_tiled<BT, HINT>(D, tb, cpar, upar, u, r, w, v, pkeep, pstream)) {
                    aborted = true;
                    break;
                }
            }
            unsigned int fn = (!TILED && !fixed && t0 < N) ? flag[t0] : 0u;
            for (int n = TILED ? N : t0; n < N; n += T) {
                // the next node's flags load while this node's row runs
                const unsigned int f = fn;
                fn = (!fixed && n + T < N) ? flag[n + T] : 0u;
                const NbrOff o = nbr_offsets(nx, nxy, wrap, f);
                // fixed offsets: no mask, see the symmetric stencils' layout
                const float acc = HINT ? row32_sym_pol(A, cs, u, n, o, exist_flags(f, wrap), pstream, pkeep)
                                       : row32_sym<true>(A, cs, u, n, o, exist_flags(f, wrap));
                stv(w + n, acc);
                const float rn = ldv(r + n), un = ldv(u + n);
                v[0] = fmaf(rn, un, v[0]);
                v[1] = fmaf(un, acc, v[1]);
                v[2] = fmaf(rn, rn, v[2]);
            }
            publish<3>(v, part, G, S.blk);
            if (!grid_barrier(bcount, target, G, &D.status)) {
                aborted = true;
                break;
            }
            if (threadIdx.x < 32) {
                float tt[3];
                gather<3>(part, G, tt);
                if (threadIdx.x == 0) {
                    if (!first) ++sc_it;
                    const float gam = tt[0], rr = tt[2];
                    sc_gam = gam;
                    sc_rr = rr;
                    const bool nan = !(tt[0] == tt[0] && tt[1] == tt[1] && tt[2] == tt[2]);
                    sc_nan = nan ? 1 : 0;
                    const int done = (nan || rr <= sc_stop || sc_it >= D.max_iter) ? 1 : 0;
                    if (!done) {
                        const float b = first ? 0.f : gam / sc_gam_old;
                        const float a = first ? gam / tt[1] : gam / (tt[1] - b * gam / sc_alpha_old);
                        sc_beta = b;
                        sc_alpha = a;
                        sc_gam_old = gam;
                        sc_alpha_old = a;
                    }
                    sc_done = done;
                }
            }
            __syncthreads();
            if (sc_done) break;
            alpha = sc_alpha;
            beta = sc_beta;
            first = false;
        }
        if (aborted) break;
        // the sweep's correction u += delta (float-float), node by node
        correct_ff_nodes(D, t0, T);
        if (!grid_barrier(bcount, target, G, &D.status)) break;  // neighbours' u below
        // ---- the sweep's residual and the next inner solve's start
        {
            float vf[4];
            resid_ff_nodes(D, t0, T, vf);
            publish<4>(vf, part, G, S.blk);
        }
        if (!grid_barrier(bcount, target, G, &D.status)) break;
        if (threadIdx.x < 32) {
            float tt[4];
            gather<4>(part, G, tt);
            if (threadIdx.x == 0) {
                sc_itsum += sc_it;
                sc_sweeps += 1;
                const double bb = tt[0], rr = tt[1];
                const bool nan = !(rr == rr);
                const bool conv = !nan && rr <= D.tol * D.tol * bb;
                const bool more = !conv && !nan && sc_sweeps < D.max_sweeps;
                // the next inner solve's stop: (0.9 tol ||b||)^2 in float
                // units, or the float floor inner_tol^2 x its first r . r
                const double ns2 = (double)D.nscale * (double)D.nscale;
                const double target2 = 0.81 * D.tol * D.tol * (bb / ns2);
                const double floor2 = D.inner_tol * D.inner_tol * (double)tt[3];
                sc_stop = (float)(target2 > floor2 ? target2 : floor2);
                sc_more = more ? 1 : 0;
                if (S.blk == 0) {
                    // the step's figures (block 0 only; the other blocks
                    // read none of these fields)
                    D.bb = bb;
                    D.relres = bb > 0.0 ? sqrt(rr / bb) : sqrt(rr);
                    D.rr0 = tt[3];
                    D.rr = tt[3];
                    D.rz = tt[2];
                    D.sweeps = sc_sweeps;
                    D.it = sc_it;
                    D.it_total += sc_it;
                    if (nan && D.status == EP_OK) D.status = EP_ENAN;
                    if (sc_nan && D.status == EP_OK) D.status = EP_ENAN;
                    if (!conv && !more && !nan && D.status == EP_OK) D.status = EP_ENOCONV;
                    if (!more) {
                        D.f_outer = 0;
                        end_of_step(D);
                    }
                }
            }
        }
        __syncthreads();
        if (!sc_more) break;
    }
}

// Self-test of the bounded wait: one block enters a barrier of a grid of
// two, whose other block never comes (a flag that nothing sets).  The spin
// gives up after spin_limit naps, records EP_ETIMEOUT in *status and the
// kernel returns; nothing faults and the context stays usable.
__global__ void k_barrier_probe(unsigned long long* count, int* status, long long spin_limit) {
    unsigned long long target = 0ull;
    (void)grid_barrier(count, target, 2, status, spin_limit);
}

cudaError_t barrier_timeout_probe(int* status_out) {
    void* mem = nullptr;
    cudaError_t e = cudaMalloc(&mem, 64);
    if (e != cudaSuccess) return e;
    unsigned long long* count = static_cast<unsigned long long*>(mem);
    int* status = reinterpret_cast<int*>(static_cast<char*>(mem) + 32);
    e = cudaMemset(mem, 0, 64);
    if (e == cudaSuccess) {
        k_barrier_probe<<<1, 32>>>(count, status, 1ll << 16);
        e = cudaGetLastError();
    }
    if (e == cudaSuccess) e = cudaDeviceSynchronize();
    if (e == cudaSuccess) e = cudaMemcpy(status_out, status, sizeof(int), cudaMemcpyDeviceToHost);
    cudaFree(mem);
    return e;
}

// Blocks of the persistent solve (1024 threads) that fit on one SM at once.
int pcg_blocks_per_sm() {
    int occ = 0;
    const cudaError_t e =
        cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve32_stencil<1024, 1, false, false>, 1024, 0);
    return e == cudaSuccess ? occ : 0;
}

int pcg_threads_of() { return 1024; }

// The tiled solve's shared memory (smem bytes) set on both variants, and
// whether a block of it fits on an SM (cooperative launches need every block
// resident).  Called once, at create.
cudaError_t pcg_tiled_prepare(size_t smem, int* fits) {
    *fits = 0;
    cudaError_t e = cudaFuncSetAttribute(k_solve32_stencil<1024, 1, true, true>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e == cudaSuccess)
        e = cudaFuncSetAttribute(k_solve32_stencil<1024, 1, false, true>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                 (int)smem);
    int occ = 0;
    if (e == cudaSuccess)
        e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&occ, k_solve32_stencil<1024, 1, true, true>, 1024, smem);
    *fits = occ >= 1;
    return e;
}

template <int BT, int MINB, bool HINT, bool TILED>
cudaError_t launch_solve(const Batch& B, int grid, size_t smem, cudaStream_t s) {
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(BT);
    cfg.dynamicSmemBytes = TILED ? smem : 0;
    cfg.stream = s;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    return cudaLaunchKernelEx(&cfg, k_solve32_stencil<BT, MINB, HINT, TILED>, B);
}

// hint: the solve's working set exceeds L2 (L2 eviction-priority policies)
cudaError_t launch_pcg32_batch(const Batch& B, int grid, int hint, cudaStream_t s) {
    return hint ? launch_solve<1024, 1, true, false>(B, grid, 0, s) : launch_solve<1024, 1, false, false>(B, grid, 0, s);
}

// tiled: the tile plan in the descriptor, grid = tile_jt x tile_kr blocks
cudaError_t launch_pcg32(Dev* d, const Dev& h, int grid, int tiled, int hint, cudaStream_t s) {
    const Batch B = single_batch(d);
    if (tiled) {
        const size_t smem = tiled_smem_bytes(h.tile_l, h.NX);
        return hint ? launch_solve<1024, 1, true, true>(B, grid, smem, s)
                    : launch_solve<1024, 1, false, true>(B, grid, smem, s);
    }
    return hint ? launch_solve<1024, 1, true, false>(B, grid, 0, s) : launch_solve<1024, 1, false, false>(B, grid, 0, s);
}

// Dynamic shared memory a block of the tiled solve may take: the opt-in
// maximum per block less the kernel's static shared memory (either variant's).
size_t tiled_smem_max() {
    int dev = 0, optin = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&optin, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev) != cudaSuccess) return 0;
    cudaFuncAttributes a1{}, a2{};
    if (cudaFuncGetAttributes(&a1, k_solve32_stencil<1024, 1, true, true>) != cudaSuccess) return 0;
    if (cudaFuncGetAttributes(&a2, k_solve32_stencil<1024, 1, false, true>) != cudaSuccess) return 0;
    const size_t st = a1.sharedSizeBytes > a2.sharedSizeBytes ? a1.sharedSizeBytes : a2.sharedSizeBytes;
    return (size_t)optin > st ? (size_t)optin - st : 0;
}

// Tile plan of the tiled apply for a mesh of NX x NY x NZ nodes on `sms`
// SMs (one 1024-thread block each), shared memory per block at most
// smem_max: among tile heights BY (rows of j) whose staging buffers fit, the
// one with the fewest staged floats per block and apply -- planes per block
// times (BY + 2) NX, the halo rows included -- with sms / ceil(NY / BY)
// ranges of k per column of tiles.  Returns false when no height fits.
// *cost: that figure over the ideal N / sms.
bool plan_tiles(int NX, int NY, int NZ, int sms, size_t smem_max, int* by, int* jt, int* kr, int* l,
                double* cost) {
    double best = 0.0;
    bool found = false;
    for (int BY = 1; BY <= NY; ++BY) {
        const int JT = (NY + BY - 1) / BY;
        if (JT > sms) continue;
        int KR = sms / JT;
        if (KR > NZ) KR = NZ;
        // the tile's rows and two halo rows, a float of slack at either
        // end, up to three of alignment before and after
        const int L = ((BY + 2) * NX + 8 + 3) / 4 * 4;
        if (tiled_smem_bytes(L, NX) > smem_max) break;  // grows with BY
        const int planes = (NZ + KR - 1) / KR;
        const double c = (double)planes * (double)(BY + 2) * NX;
        if (!found || c < best) {
            found = true;
            best = c;
            *by = BY;
            *jt = JT;
            *kr = KR;
            *l = L;
        }
    }
    if (found) *cost = best / ((double)NX * NY * NZ / sms);
    return found;
}

}  // namespace epk
