// Spatial partition of the event space (§Partitioning the World) and the
// per-sweep boundary shift (§Chromatic MH with Dynamic Coloring).
//
// A sweep starts by re-binning every event into the cells of the shifted grid:
//   rebin_count   one block per new cell counts the events that fall in it;
//                 the old cells that can feed a new cell are its 3 x 3
//                 neighbourhood, because the two grids differ by less than
//                 one cell side along each axis;
//   rebin_scan    one block: exclusive scan of (count + k births of slack)
//                 over cells -> slices of the new store; colour lists of the
//                 live cells (cells with a non-empty intersection with the
//                 domain), each in cell-index order;
//   rebin_gather  one block per new cell collects its events and writes them
//                 sorted by event id, the canonical order every region uses.
#include <cuda_runtime.h>

#include "cmh_common.cuh"

namespace cmh {

namespace {

constexpr int kRebinThreads = 128;

__device__ __forceinline__ bool cell_live(const Geo& g, double sx, double sy, int c) {
    double r[4];
    cell_rect(g, sx, sy, c, r);
    return r[1] > r[0] && r[3] > r[2];
}

// iterate the candidate old events of new cell c: the 3 x 3 old cells around
// c, or (init_n >= 0) the flat list [0, init_n) of store `old`
template <typename F>
__device__ __forceinline__ void for_candidates(const Geo& g, const Store& old, int c, int init_n, F&& f) {
    if (init_n >= 0) {
        for (int base = 0; base < init_n; base += blockDim.x) f(base + (int)threadIdx.x, base + (int)threadIdx.x < init_n);
        return;
    }
    const int ix = c % g.ncx, iy = c / g.ncx;
    for (int jy = iy - 1; jy <= iy + 1; ++jy) {
        if (jy < 0 || jy >= g.ncy) continue;
        for (int jx = ix - 1; jx <= ix + 1; ++jx) {
            if (jx < 0 || jx >= g.ncx) continue;
            const int oc = jy * g.ncx + jx;
            const int s0 = old.start[oc], n = old.count[oc];
            for (int base = 0; base < n; base += blockDim.x) {
                const int i = base + (int)threadIdx.x;
                f(s0 + i, i < n);
            }
        }
    }
}

__global__ void __launch_bounds__(kRebinThreads) rebin_count(Geo g, Dev d, int init_n) {
    if (*d.status) return;
    const long long sweep = *d.sweep;
    double sx, sy;
    sweep_shift(g, sweep, &sx, &sy);
    if (blockIdx.x == 0 && threadIdx.x == 0) {
        d.shift[0] = sx;
        d.shift[1] = sy;
    }
    const Store old = d.st[(sweep + 1) & 1];
    const int c = blockIdx.x;
    int cnt = 0;
    if (cell_live(g, sx, sy, c)) {
        for_candidates(g, old, c, init_n, [&](int idx, bool ok) {
            if (ok && cell_of(g, sx, sy, old.x[idx], old.y[idx]) == c) ++cnt;
        });
    }
    __shared__ int s_cnt;
    if (threadIdx.x == 0) s_cnt = 0;
    __syncthreads();
    for (int o = 16; o > 0; o >>= 1) cnt += __shfl_xor_sync(0xffffffffu, cnt, o);
    if ((threadIdx.x & 31) == 0 && cnt) atomicAdd(&s_cnt, cnt);
    __syncthreads();
    if (threadIdx.x == 0) d.fill[c] = s_cnt;
}

// live cells form a rectangle in index space; the colour lists hold them in
// cell-index order: rank of (ix, iy) among live cells of the same colour
__device__ __forceinline__ bool x_live(const Geo& g, double s, int ix) {
    double a = __dadd_rn(s, __dmul_rn((double)(ix - 1), g.L));
    double b = __dadd_rn(s, __dmul_rn((double)ix, g.L));
    if (a < 0.0) a = 0.0;
    if (b > g.W) b = g.W;
    return b > a;
}

__global__ void __launch_bounds__(1024) rebin_scan(Geo g, Dev d) {
    if (*d.status) return;
    const long long sweep = *d.sweep;
    const Store nw = d.st[sweep & 1];
    const double sx = d.shift[0], sy = d.shift[1];
    __shared__ long long s_carry, s_events;
    __shared__ long long s_warp[32];
    if (threadIdx.x == 0) { s_carry = 0; s_events = 0; }
    __syncthreads();
    const int lane = threadIdx.x & 31, wid = threadIdx.x >> 5, nwarp = blockDim.x >> 5;
    for (int base = 0; base < g.n_cells; base += blockDim.x) {
        const int c = base + threadIdx.x;
        long long v = 0;
        int cnt = 0;
        bool live = false;
        if (c < g.n_cells) {
            cnt = d.fill[c];
            live = x_live(g, sx, c % g.ncx) && x_live(g, sy, c / g.ncx);
            v = cnt + (live ? g.k : 0);
        }
        // block inclusive scan of v
        long long x = v;
        for (int o = 1; o < 32; o <<= 1) {
            long long y = __shfl_up_sync(0xffffffffu, x, o);
            if (lane >= o) x += y;
        }
        if (lane == 31) s_warp[wid] = x;
        long long ev = cnt;
        for (int o = 16; o > 0; o >>= 1) ev += __shfl_xor_sync(0xffffffffu, ev, o);
        if (lane == 0) atomicAdd((unsigned long long*)&s_events, (unsigned long long)ev);
        __syncthreads();
        if (wid == 0) {
            long long w = lane < nwarp ? s_warp[lane] : 0;
            for (int o = 1; o < 32; o <<= 1) {
                long long y = __shfl_up_sync(0xffffffffu, w, o);
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
    // colour lists
    const int P = g.period;
    for (int c = threadIdx.x; c < g.n_cells; c += blockDim.x) {
        const int ix = c % g.ncx, iy = c / g.ncx;
        if (!(x_live(g, sx, ix) && x_live(g, sy, iy))) continue;
        int rx = 0, nx = 0, ry = 0;
        for (int j = ix % P; j < g.ncx; j += P) {
            if (!x_live(g, sx, j)) continue;
            if (j < ix) ++rx;
            ++nx;
        }
        for (int j = iy % P; j < iy; j += P)
            if (x_live(g, sy, j)) ++ry;
        const int col = (ix % P) + P * (iy % P);
        d.colour_cells[col * g.max_rpc + ry * nx + rx] = c;
    }
    for (int col = threadIdx.x; col < g.n_colours; col += blockDim.x) {
        const int cx = col % P, cy = col / P;
        int nx = 0, ny = 0;
        for (int j = cx; j < g.ncx; j += P) nx += x_live(g, sx, j);
        for (int j = cy; j < g.ncy; j += P) ny += x_live(g, sy, j);
        d.colour_count[col] = nx * ny;
    }
}

__global__ void __launch_bounds__(kRebinThreads) rebin_gather(Geo g, Dev d, int init_n) {
    if (*d.status) return;
    const long long sweep = *d.sweep;
    const Store old = d.st[(sweep + 1) & 1];
    const Store nw = d.st[sweep & 1];
    const double sx = d.shift[0], sy = d.shift[1];
    const int c = blockIdx.x;
    const int n = nw.count[c];
    if (n == 0) return;
    if (n > g.ev_cap) {
        if (threadIdx.x == 0) latch(d.status, CMH_ERR_CAPACITY);
        return;
    }
    extern __shared__ __align__(16) unsigned char smem[];
    double* bx = (double*)smem;
    double* by = bx + g.ev_cap;
    double* bt = by + g.ev_cap;
    double* bm = bt + g.ev_cap;
    unsigned long long* bid = (unsigned long long*)(bm + g.ev_cap);
    __shared__ int s_pos;
    if (threadIdx.x == 0) s_pos = 0;
    __syncthreads();
    for_candidates(g, old, c, init_n, [&](int idx, bool ok) {
        if (ok && cell_of(g, sx, sy, old.x[idx], old.y[idx]) == c) {
            const int p = atomicAdd(&s_pos, 1);
            if (p < g.ev_cap) {
                bx[p] = old.x[idx];
                by[p] = old.y[idx];
                bt[p] = old.t[idx];
                bm[p] = old.m[idx];
                bid[p] = old.id[idx];
            }
        }
    });
    __syncthreads();
    // rank by id (ids are unique) and write in id order
    const int s0 = nw.start[c];
    for (int i = threadIdx.x; i < n; i += blockDim.x) {
        const unsigned long long me = bid[i];
        int r = 0;
        for (int j = 0; j < n; ++j) r += bid[j] < me;
        nw.x[s0 + r] = bx[i];
        nw.y[s0 + r] = by[i];
        nw.t[s0 + r] = bt[i];
        nw.m[s0 + r] = bm[i];
        nw.id[s0 + r] = me;
    }
}

}  // namespace

cudaError_t launch_rebin(const Geo& g, const Dev& d, int init_n, cudaStream_t s, int* launches) {
    rebin_count<<<g.n_cells, kRebinThreads, 0, s>>>(g, d, init_n);
    rebin_scan<<<1, 1024, 0, s>>>(g, d);
    const size_t smem = (size_t)g.ev_cap * (4 * sizeof(double) + sizeof(unsigned long long));
    rebin_gather<<<g.n_cells, kRebinThreads, smem, s>>>(g, d, init_n);
    if (launches) *launches += 3;
    return cudaGetLastError();
}

}  // namespace cmh
