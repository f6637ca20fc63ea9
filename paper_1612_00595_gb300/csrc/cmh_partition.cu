// Spatial partition of the event space (§Partitioning the World) and the
// per-sweep boundary shift (§Chromatic MH with Dynamic Coloring).
//
// A sweep starts by re-binning every event into the cells of the shifted grid:
//   rebin_assign  one warp per old cell (or one thread per event of the
//                 initial flat list) computes the new cell of each event and
//                 counts it into fill[] with an atomic add;
//   rebin_scan    one block: exclusive scan of (count + k births of slack)
//                 over cells -> slices of the new store (fill is cleared for
//                 the next sweep); colour lists of the live cells (cells with
//                 a non-empty intersection with the domain), each in
//                 cell-index order;
//   rebin_gather  one warp per new cell collects its events from the 3 x 3
//                 old cells around it (the two grids differ by less than one
//                 cell side along each axis), by their new-cell index, and
//                 writes them sorted by event id, the canonical order every
//                 region uses (with latent arrival times, each event's row
//                 of offsets with it).
// Only rebin_assign evaluates the cell index of a coordinate; the exact
// float64 form of floor((x - s) / L) runs only when a float32 estimate lies
// within 1e-3 of an integer.
#include <cuda_runtime.h>

#include <algorithm>

#include "cmh_common.cuh"

namespace cmh {

namespace {

constexpr unsigned FULL = 0xffffffffu;
constexpr int kRebinThreads = 256;
constexpr int kWarpsPerBlock = kRebinThreads / 32;
constexpr int kAxisMax = 1024;   // cells per axis (the host keeps ncx * ncy <= 2^20)
constexpr int kMaxPeriod = 4;    // colour period per axis (the host keeps P^2 <= kMaxColours)

// cell index along one axis, floor((x - s) / L) + 1 as its float64 definition
// gives it.  The float32 quotient is within |q| 2^-22 of the float64 one;
// away from integers by more than 1e-3 (|q| <= 1024 cells) its floor is the
// same, otherwise the float64 division decides.
__device__ __forceinline__ int cell_axis_fast(const Geo& g, double x, double s) {
    const double dd = __dsub_rn(x, s);
    const float q = (float)dd * g.invL_f;
    const float fl = floorf(q);
    if (q - fl > 1e-3f && fl + 1.f - q > 1e-3f) return (int)fl + 1;
    return cell_axis(x, s, g.L);
}

__device__ __forceinline__ int cell_of_fast(const Geo& g, double sx, double sy, double x, double y) {
    const int ix = cell_axis_fast(g, x, sx), iy = cell_axis_fast(g, y, sy);
    if (ix < 0 || ix >= g.ncx || iy < 0 || iy >= g.ncy) return -1;
    return iy * g.ncx + ix;
}

// block `blk` of an instance's rebin_assign
__device__ __forceinline__ void rebin_assign_body(const Geo& g, const Dev& d, int init_n, int blk) {
    if (*d.status) return;
    const long long sweep = *d.sweep;
    double sx, sy;
    sweep_shift(g, sweep, &sx, &sy);
    if (blk == 0 && threadIdx.x == 0) {
        d.shift[0] = sx;
        d.shift[1] = sy;
    }
    const Store old = d.st[(sweep + 1) & 1];
    auto assign = [&](int pos) {
        const int c = cell_of_fast(g, sx, sy, old.x[pos], old.y[pos]);
        d.ncell[pos] = c;
        if (c >= 0)
            atomicAdd(&d.fill[c], 1);
        else
            latch(d.status, CMH_ERR_GEOMETRY);   // an event outside the domain
    };
    if (init_n >= 0) {
        const int i = blk * blockDim.x + threadIdx.x;
        if (i < init_n) assign(i);
        return;
    }
    const int oc = blk * kWarpsPerBlock + (int)(threadIdx.x >> 5);
    if (oc >= g.n_cells) return;
    const int s0 = old.start[oc], n = old.count[oc];
    for (int i = threadIdx.x & 31; i < n; i += 32) assign(s0 + i);
}

// is index i along an axis (shift s) a live cell: [s + (i-1) L, s + i L) meets [0, W)
__device__ __forceinline__ bool axis_live(const Geo& g, double s, int i) {
    double a = __dadd_rn(s, __dmul_rn((double)(i - 1), g.L));
    double b = __dadd_rn(s, __dmul_rn((double)i, g.L));
    if (a < 0.0) a = 0.0;
    if (b > g.W) b = g.W;
    return b > a;
}

__device__ __forceinline__ void rebin_scan_body(const Geo& g, const Dev& d) {
    if (*d.status) return;
    const long long sweep = *d.sweep;
    const Store nw = d.st[sweep & 1];
    const double sx = d.shift[0], sy = d.shift[1];
    const int P = g.period;
    __shared__ long long s_carry, s_events;
    __shared__ long long s_warp[32];
    __shared__ unsigned char s_live[2][kAxisMax];
    __shared__ int s_rank[2][kAxisMax];     // rank among the live indices of the same residue mod P
    __shared__ int s_num[2][kMaxPeriod];    // live indices of each residue
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    if (threadIdx.x == 0) {
        s_carry = 0;
        s_events = 0;
    }
    for (int i = threadIdx.x; i < g.ncx; i += blockDim.x) s_live[0][i] = axis_live(g, sx, i);
    for (int i = threadIdx.x; i < g.ncy; i += blockDim.x) s_live[1][i] = axis_live(g, sy, i);
    __syncthreads();
    if (threadIdx.x < 2 * P) {
        const int ax = threadIdx.x / P, r = threadIdx.x % P, n = ax ? g.ncy : g.ncx;
        int cnt = 0;
        for (int i = r; i < n; i += P) {
            s_rank[ax][i] = cnt;
            cnt += s_live[ax][i];
        }
        s_num[ax][r] = cnt;
    }
    __syncthreads();
    for (int base = 0; base < g.n_cells; base += blockDim.x) {
        const int c = base + threadIdx.x;
        long long v = 0;
        int cnt = 0;
        if (c < g.n_cells) {
            cnt = d.fill[c];
            d.fill[c] = 0;
            v = cnt + ((s_live[0][c % g.ncx] && s_live[1][c / g.ncx]) ? g.k : 0);
        }
        // block inclusive scan of v
        long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(FULL, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[wid] = x;
        long long ev = cnt;
        for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(FULL, ev, o);
        if (lane == 0) atomicAdd((unsigned long long*)&s_events, (unsigned long long)ev);
        __syncthreads();
        if (wid == 0) {
            long long w = lane < nwarp ? s_warp[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(FULL, w, o);
                if (lane >= o) w += y;
            }
            if (lane < nwarp) s_warp[lane] = w;
        }
        __syncthreads();
        const long long excl = s_carry + (wid ? s_warp[wid - 1] : 0) + x - v;
        if (c < g.n_cells) {
            nw.start[c] = (int)excl;
            nw.count[c] = cnt;
            nw.cap[c] = (int)v;
        }
        __syncthreads();
        if (threadIdx.x == blockDim.x - 1) s_carry = excl + v;
        __syncthreads();
    }
    if (threadIdx.x == 0) {
        if (s_carry > g.store_cap || s_events > g.max_events) latch(d.status, CMH_ERR_CAPACITY);
        *nw.total = (int)s_events;
    }
    // colour lists: live cell (ix, iy) has colour (ix mod P) + P (iy mod P) and
    // position (rank of iy) x (live columns of its residue) + (rank of ix)
    for (int c = threadIdx.x; c < g.n_cells; c += blockDim.x) {
        const int ix = c % g.ncx, iy = c / g.ncx;
        if (!(s_live[0][ix] && s_live[1][iy])) {
            d.cell_col[c] = -1;
            continue;
        }
        const int col = (ix % P) + P * (iy % P);
        d.cell_col[c] = col;
        d.colour_cells[col * g.max_rpc + s_rank[1][iy] * s_num[0][ix % P] + s_rank[0][ix]] = c;
    }
    for (int col = threadIdx.x; col < g.n_colours; col += blockDim.x)
        d.colour_count[col] = s_num[0][col % P] * s_num[1][col / P];
    // the queue of the persistent sweep: regions in colour order
    if (threadIdx.x == 0) {
        int off = 0;
        for (int col = 0; col < g.n_colours; ++col) {
            d.colour_off[col] = off;
            off += s_num[0][col % P] * s_num[1][col / P];
        }
        d.colour_off[g.n_colours] = off;
        *d.queue = 0;
    }
}

__device__ __forceinline__ void rebin_gather_body(const Geo& g, const Dev& d, int init_n, int wpb, int blk,
                                                  unsigned char* smem) {
    if (*d.status) return;
    const long long sweep = *d.sweep;
    const Store old = d.st[(sweep + 1) & 1];
    const Store nw = d.st[sweep & 1];
    const int lane = threadIdx.x & 31, w = threadIdx.x >> 5;
    const int c = blk * wpb + w;
    if (c >= g.n_cells) return;
    const int n = nw.count[c];
    if (n == 0) return;
    if (n > g.ev_cap) {
        if (lane == 0) latch(d.status, CMH_ERR_CAPACITY);
        return;
    }
    unsigned long long* bid = (unsigned long long*)smem + (size_t)w * g.ev_cap;
    int* bpos = (int*)((unsigned long long*)smem + (size_t)wpb * g.ev_cap) + (size_t)w * g.ev_cap;
    const unsigned lt = (1u << lane) - 1u;
    int got = 0;
    auto collect = [&](int s0, int cnt) {
        for (int i0 = 0; i0 < cnt; i0 += 32) {
            const int i = i0 + lane;
            const bool hit = i < cnt && d.ncell[s0 + i] == c;
            const unsigned bal = __ballot_sync(FULL, hit);
            if (hit) {
                const int p = got + __popc(bal & lt);
                if (p < g.ev_cap) {
                    bpos[p] = s0 + i;
                    bid[p] = old.id[s0 + i];
                }
            }
            got += __popc(bal);
        }
    };
    if (init_n >= 0) {
        collect(0, init_n);
    } else {
        // the (up to) nine old cells around c: lanes 0..8 read their slices
        // at once, then the warp scans their events as one flat range (the
        // collection order does not matter: the events are ranked by id)
        const int ix = c % g.ncx, iy = c / g.ncx;
        int s0 = 0, cnt = 0;
        if (lane < 9) {
            const int jx = ix - 1 + lane % 3, jy = iy - 1 + lane / 3;
            if (jx >= 0 && jx < g.ncx && jy >= 0 && jy < g.ncy) {
                const int oc = jy * g.ncx + jx;
                s0 = old.start[oc];
                cnt = old.count[oc];
            }
        }
        int incl = cnt;   // inclusive prefix of the nine counts
        for (int o = 1; o < 16; o <<= 1) {
            const int v = __shfl_up_sync(FULL, incl, o);
            if (lane >= o) incl += v;
        }
        const int total = __shfl_sync(FULL, incl, 8);
        for (int i0 = 0; i0 < total; i0 += 32) {
            const int i = i0 + lane, ic = min(i, total - 1);   // every lane shuffles
            int q = 0;   // the cell holding flat index ic: the first whose prefix exceeds it
#pragma unroll
            for (int u = 0; u < 8; ++u) q += ic >= __shfl_sync(FULL, incl, u) ? 1 : 0;
            const int bq = __shfl_sync(FULL, incl, q > 0 ? q - 1 : 0);
            const int src = __shfl_sync(FULL, s0, q) + (ic - (q > 0 ? bq : 0));
            const bool hit = i < total && d.ncell[src] == c;
            const unsigned bal = __ballot_sync(FULL, hit);
            if (hit) {
                const int p = got + __popc(bal & lt);
                if (p < g.ev_cap) {
                    bpos[p] = src;
                    bid[p] = old.id[src];
                }
            }
            got += __popc(bal);
        }
    }
    __syncwarp();
    if (got != n) {   // counted and collected events disagree: not expected
        if (lane == 0) latch(d.status, CMH_ERR_GEOMETRY);
        return;
    }
    // rank by id (ids are unique) and write in id order
    const int s0 = nw.start[c];
    for (int i = lane; i < n; i += 32) {
        const unsigned long long me = bid[i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += bid[j] < me;
        const int src = bpos[i];
        nw.x[s0 + r] = old.x[src];
        nw.y[s0 + r] = old.y[src];
        nw.t[s0 + r] = old.t[src];
        nw.m[s0 + r] = old.m[src];
        nw.id[s0 + r] = me;
        if (nw.off)   // latent arrival offsets travel with their event
            for (int j = 0; j < g.n_st; ++j)
                nw.off[(size_t)(s0 + r) * g.n_st + j] = old.off[(size_t)src * g.n_st + j];
    }
}

__global__ void __launch_bounds__(kRebinThreads) rebin_assign(const __grid_constant__ Geo g,
                                                              const __grid_constant__ Dev d, int init_n) {
    rebin_assign_body(g, d, init_n, blockIdx.x);
}

__global__ void __launch_bounds__(1024) rebin_scan(const __grid_constant__ Geo g, const __grid_constant__ Dev d) {
    rebin_scan_body(g, d);
}

__global__ void __launch_bounds__(kRebinThreads) rebin_gather(const __grid_constant__ Geo g,
                                                              const __grid_constant__ Dev d, int init_n, int wpb) {
    extern __shared__ __align__(16) unsigned char smem[];
    rebin_gather_body(g, d, init_n, wpb, blockIdx.x, smem);
}

// ---- a batch of independent instances: the same bodies, one instance per
// block range (blk_off[i] .. blk_off[i+1]) or per block ----------------------
__device__ __forceinline__ int instance_of_block(const int* blk_off, int n_inst, int b) {
    int lo = 0, hi = n_inst - 1;   // largest i with blk_off[i] <= b
    while (lo < hi) {
        const int mid = (lo + hi + 1) >> 1;
        if (blk_off[mid] <= b) lo = mid; else hi = mid - 1;
    }
    return lo;
}

__global__ void __launch_bounds__(kRebinThreads) rebin_assign_batch(const Geo* G, const Dev* D, const int* blk_off,
                                                                    int n_inst) {
    const int i = instance_of_block(blk_off, n_inst, blockIdx.x);
    rebin_assign_body(G[i], D[i], -1, blockIdx.x - blk_off[i]);
}

__global__ void __launch_bounds__(1024) rebin_scan_batch(const Geo* G, const Dev* D) {
    rebin_scan_body(G[blockIdx.x], D[blockIdx.x]);
}

__global__ void __launch_bounds__(kRebinThreads) rebin_gather_batch(const Geo* G, const Dev* D, const int* blk_off,
                                                                    int n_inst) {
    extern __shared__ __align__(16) unsigned char smem[];
    const int i = instance_of_block(blk_off, n_inst, blockIdx.x);
    rebin_gather_body(G[i], D[i], -1, kWarpsPerBlock, blockIdx.x - blk_off[i], smem);
}

}  // namespace

namespace {

// warps (new cells) per rebin_gather block: each holds ev_cap ids and positions
int gather_warps(const Geo& g) { return g.ev_cap <= 512 ? kWarpsPerBlock : 1; }

size_t gather_smem(const Geo& g) {
    return (size_t)gather_warps(g) * g.ev_cap * (sizeof(unsigned long long) + sizeof(int));
}

}  // namespace

cudaError_t prepare_rebin(const Geo& g) {
    return raise_smem_limit((const void*)rebin_gather, gather_smem(g));
}

// blocks of rebin_assign / rebin_gather for one instance in a batch
int rebin_blocks(const Geo& g) { return (g.n_cells + kWarpsPerBlock - 1) / kWarpsPerBlock; }

size_t rebin_batch_smem(int max_ev_cap) {
    return (size_t)kWarpsPerBlock * max_ev_cap * (sizeof(unsigned long long) + sizeof(int));
}

cudaError_t prepare_rebin_batch(int max_ev_cap) {
    return raise_smem_limit((const void*)rebin_gather_batch, rebin_batch_smem(max_ev_cap));
}

cudaError_t launch_rebin_batch(const Geo* G, const Dev* D, const int* blk_off, int n_inst, int n_blocks,
                               int max_ev_cap, cudaStream_t s) {
    const size_t smem = rebin_batch_smem(max_ev_cap);
    rebin_assign_batch<<<n_blocks, kRebinThreads, 0, s>>>(G, D, blk_off, n_inst);
    rebin_scan_batch<<<n_inst, 1024, 0, s>>>(G, D);
    rebin_gather_batch<<<n_blocks, kRebinThreads, smem, s>>>(G, D, blk_off, n_inst);
    return cudaGetLastError();
}

cudaError_t launch_rebin(const Geo& g, const Dev& d, int init_n, cudaStream_t s, int* launches) {
    const int assign_blocks = init_n >= 0 ? std::max(1, (init_n + kRebinThreads - 1) / kRebinThreads)
                                          : (g.n_cells + kWarpsPerBlock - 1) / kWarpsPerBlock;
    rebin_assign<<<assign_blocks, kRebinThreads, 0, s>>>(g, d, init_n);
    rebin_scan<<<1, 1024, 0, s>>>(g, d);
    const int wpb = gather_warps(g);
    rebin_gather<<<(g.n_cells + wpb - 1) / wpb, 32 * wpb, gather_smem(g), s>>>(g, d, init_n, wpb);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

}  // namespace cmh
