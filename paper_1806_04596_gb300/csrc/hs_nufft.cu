// De-gridding G_l and gridding G_l^H with the 8 x 8 Kaiser-Bessel window (Sec.
// 2.1: each row of G_l holds the interpolation kernel of one visibility), all
// channels in one launch, fused with the data-fidelity dual update of
// Algorithm 2 steps 10-12.
//
// Kernel values are computed on the fly: phi(m + f) for the unit piece m is a
// fitted polynomial in s = 2 f - 1 (FP32: 9 coefficients, error 7e-9 of phi(0);
// FP64: 14 coefficients, 6e-15). De-gridding evaluates one piece per lane (8
// independent Horner chains at the same s); gridding evaluates the 8 taps of an
// axis in one lane as 4 mirrored pairs of even/odd polynomials.
//
// De-gridding: 8 lanes per visibility, lane j owns window column j and walks
// the 8 rows (coalesced 64-byte row segments), then the 8 lanes reduce by
// shuffles. Visibilities are processed in the plan's tile-sorted order so
// neighbouring lanes touch neighbouring grid cells.
//
// Gridding writes every output cell exactly once, so the grid needs no zeroing
// pass and no global atomics, and sums in a fixed order (deterministic).
// Default kernel on grids of at least 64 x 64 cells: the register sweep
// (k_grid_sweep, below). Smaller grids: one CTA per (channel, 32 x 32 tile)
// consumes the tile's list of overlapping windows, every warp adding groups of
// 4 mutually non-overlapping windows into its private copy of the tile in
// shared memory, the copies combined in a fixed order. HS_PLAN_COMPENSATED
// kernel: the same tiles, one window per warp at a time, with Kahan-compensated
// FP32 sums.
#include "hs_device.cuh"
#include "hs_internal.h"

namespace hs {

template <typename R> struct VisCoord;
template <> struct VisCoord<float> {
    // fixed point: cell in the high bits, fraction in the low `fb` bits
    static __device__ __forceinline__ void get(const void* c, int64_t i, const Geo& g, int& cxv,
                                               int& cyv, float& fx, float& fy) {
        const uint2 t = ((const uint2*)c)[i];
        cxv = (int)(t.x >> g.fbx);
        cyv = (int)(t.y >> g.fby);
        fx = (float)(t.x & ((1u << g.fbx) - 1u)) * __int_as_float((127 - g.fbx) << 23);
        fy = (float)(t.y & ((1u << g.fby) - 1u)) * __int_as_float((127 - g.fby) << 23);
    }
};
template <> struct VisCoord<double> {
    static __device__ __forceinline__ void get(const void* c, int64_t i, const Geo& g, int& cxv,
                                               int& cyv, double& fx, double& fy) {
        const Coord64 t = ((const Coord64*)c)[i];
        cxv = t.cx;
        cyv = t.cy;
        fx = t.fx;
        fy = t.fy;
    }
};

template <typename R> struct NufftK {
    Geo g;
    const Cx<R>* grid;
    Cx<R>* grid_out;
    const void* coords;
    const int64_t* off;
    const R* w;        // Theta (sorted) or null
    const R* u;        // U (sorted) or null
    const int* perm;   // sorted -> caller
    const R* kbc;      // 8 x NC coefficients
    // pieces 7 - m, m = 0 .. 3, split into even and odd coefficients (passed by value,
    // so a warp-uniform Horner step reads its coefficient from the parameter bank)
    R kev[4 * KB_HALF];
    R kod[4 * KB_HALF];
    // de-gridding outputs / PD inputs
    Cx<R>* out;
    Cx<R>* v;
    const Cx<R>* y;
    Cx<R>* d;
    double* part;
    int nblk_x;
    // gridding inputs
    const Cx<R>* in;
    const R* scale;
    const int64_t* tile_off;
    const int* tile_ent;
    const int* blk;    // block of every sorted visibility (data blocks), or null: one block per channel
    double* rpart;     // DOUT_PD: per-item partial ||y - Phi x~||^2 (adaptive bounds), or null
};

// ---------------------------------------------------------------- de-gridding
// Work item (built by the plan): a run of at most DEGRID_CHUNK sorted
// visibilities of one channel whose windows start in one 32 x 32 tile. The CTA
// stages the tile's (32 + 8) x (32 + 8) window region of the grid into shared
// memory with asynchronous copies (one global read per cell, wrapped), then
// interpolates every visibility from shared memory.
struct DgItem {
    int tix;      // l * ntiles + tile
    int e0, e1;   // sorted visibility range
    int slot;     // partial-sum slot (PD mode)
};
constexpr int DG_REG = GRID_TILE + 8;   // staged region side (window start offsets 0..32)
constexpr int DG_LDS = DG_REG + 2;    // even: 16-byte aligned staged rows

template <typename R> __device__ __forceinline__ void cp_async_cx(Cx<R>* dst, const Cx<R>* src) {
    const unsigned d = (unsigned)__cvta_generic_to_shared(dst);
    if constexpr (sizeof(R) == 4)
        asm volatile("cp.async.ca.shared.global [%0], [%1], 8;\n" ::"r"(d), "l"(src) : "memory");
    else
        asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
}

template <typename R, int NC, int MODE>
__global__ void __launch_bounds__(256, sizeof(R) == 4 ? 5 : 1)
    k_degrid(NufftK<R> a, const DgItem* __restrict__ items) {
    typedef Cx<R> CT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT* S = reinterpret_cast<CT*>(smem_raw);   // [DG_REG][DG_LDS]
    __shared__ double red[32];
    const DgItem it = items[blockIdx.x];
    const int ntiles = a.g.ntx * a.g.nty;
    const int l = it.tix / ntiles;
    const int t = it.tix - l * ntiles;
    const int Kx = a.g.Kx, Ky = a.g.Ky;
    const int kxm = a.g.kxm, kym = a.g.kym;
    const int ty0 = (t / a.g.ntx) * a.g.ty, tx0 = (t % a.g.ntx) * a.g.tx;
    const CT* G = a.grid + (int64_t)l * Ky * Kx;
    if constexpr (sizeof(R) == 4) {
        // FP32: 16-byte chunks of two cells (tx0 and Kx even: a chunk never straddles the wrap)
        constexpr int CPR = DG_REG / 2;   // chunks per staged row
        for (int k = threadIdx.x; k < DG_REG * CPR; k += blockDim.x) {
            const int r = k / CPR, c = 2 * (k - r * CPR);
            const unsigned d = (unsigned)__cvta_generic_to_shared(S + r * DG_LDS + c);
            const CT* src = G + (int64_t)(wrapn(ty0 + r, Ky, kym)) * Kx + (wrapn(tx0 + c, Kx, kxm));
            asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(d), "l"(src) : "memory");
        }
    } else {
        for (int k = threadIdx.x; k < DG_REG * DG_REG; k += blockDim.x) {
            const int r = k / DG_REG, c = k - r * DG_REG;
            cp_async_cx<R>(S + r * DG_LDS + c, G + (int64_t)(wrapn(ty0 + r, Ky, kym)) * Kx + (wrapn(tx0 + c, Kx, kxm)));
        }
    }
    asm volatile("cp.async.commit_group;\n" ::: "memory");
    const int lane = threadIdx.x & 31;
    const int j = lane & 7;              // window column / tap owned by this lane
    const int grp = threadIdx.x >> 3;    // 32 groups of 8 lanes
    const int gbase = lane & ~7;
    R c[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) c[k] = a.kbc[(7 - j) * NC + k];
    const int64_t beg = it.e0, end = it.e1;
    R sq = 0;   // this thread's share of ||d||^2 (few terms; FP64 only for the block sum)
    R rq = 0;   // and of ||y - Phi x~||^2 (adaptive bounds)
    // lane j of a group preloads the coordinates of the group's j-th visibility
    int pcx = 0, pcy = 0;
    R pfx = 0, pfy = 0;
    {
        const int64_t ip = beg + grp + 32 * j;
        if (ip < end) VisCoord<R>::get(a.coords, ip, a.g, pcx, pcy, pfx, pfy);
    }
    asm volatile("cp.async.wait_group 0;\n" ::: "memory");
    __syncthreads();
    // two visibilities per group and step; every lane keeps its partial of the
    // group's 8 visibilities, and one reduce-scatter over the 8 lanes leaves
    // visibility j's sum in lane j, so the epilogue runs once per group, one
    // visibility per lane
    static_assert(DEGRID_CHUNK == 8 * 32, "one visibility per lane of a group");
    CT p8[8];
#pragma unroll
    for (int k = 0; k < 8; ++k) p8[k] = cx<R>(0, 0);
#pragma unroll
    for (int it2 = 0; it2 < DEGRID_CHUNK / 32; it2 += 2) {
        if (beg + 32 * it2 >= end) break;   // uniform over the CTA
        int off[2];
        R pu[2], pv[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            const int src = gbase + it2 + h;
            const int cxv = __shfl_sync(0xffffffffu, pcx, src);
            const int cyv = __shfl_sync(0xffffffffu, pcy, src);
            const R fx = __shfl_sync(0xffffffffu, pfx, src);
            const R fy = __shfl_sync(0xffffffffu, pfy, src);
            // window start relative to the staged region: 0..32 (carry included)
            const int ox = wrapn(wrapn(cxv - 3, Kx, kxm) - tx0, Kx, kxm);
            const int oy = wrapn(wrapn(cyv - 3, Ky, kym) - ty0, Ky, kym);
            off[h] = min(oy, DG_REG - 8) * DG_LDS + min(ox, DG_REG - 8) + j;
            pu[h] = horner<R, NC>(c, (R)2 * fx - (R)1);
            pv[h] = horner<R, NC>(c, (R)2 * fy - (R)1);
        }
        CT gv[2][8];
#pragma unroll
        for (int h = 0; h < 2; ++h)
#pragma unroll
            for (int r = 0; r < 8; ++r) gv[h][r] = S[off[h] + r * DG_LDS];
        CT acc[2];
#pragma unroll
        for (int h = 0; h < 2; ++h) {
            acc[h] = cx<R>(0, 0);
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const R pvr = __shfl_sync(0xffffffffu, pv[h], gbase + r);
                acc[h].x = fma(pvr, gv[h][r].x, acc[h].x);
                acc[h].y = fma(pvr, gv[h][r].y, acc[h].y);
            }
            acc[h].x *= pu[h];
            acc[h].y *= pu[h];
        }
        p8[it2] = acc[0];
        p8[it2 + 1] = acc[1];
    }
    // reduce-scatter: at distance o, lanes with bit o set keep the upper half
#pragma unroll
    for (int o = 4; o >= 1; o >>= 1) {
        const bool up = (j & o) != 0;
#pragma unroll
        for (int k = 0; k < o; ++k) {
            const CT send = up ? p8[k] : p8[k + o];
            CT keep = up ? p8[k + o] : p8[k];
            keep.x += __shfl_xor_sync(0xffffffffu, send.x, o);
            keep.y += __shfl_xor_sync(0xffffffffu, send.y, o);
            p8[k] = keep;
        }
    }
    const CT mine = p8[0];
    {
        const int64_t i = beg + grp + 32 * j;
        if (i < end) {
            CT v = mine;
            if (a.w) v = cscale(v, a.w[i]);
            if (MODE == DOUT_CALLER) {
                a.out[a.perm[i]] = v;
            } else if (MODE == DOUT_SORTED) {
                a.out[i] = v;
            } else if (MODE == DOUT_SORTED_U) {
                a.out[i] = a.u ? cscale(v, a.u[i]) : v;
            } else {   // DOUT_PD: vbar = v + U Phi x~, d = U^{-1/2} vbar - y
                CT vb = a.v[i];
                CT dd;
                if (a.u) {
                    const R uu = a.u[i];
                    const R is = (R)1 / sqrt(uu);
                    vb.x = fma(uu, v.x, vb.x);
                    vb.y = fma(uu, v.y, vb.y);
                    dd = csub(cscale(vb, is), a.y[i]);
                } else {
                    dd = csub(cadd(vb, v), a.y[i]);
                }
                a.d[i] = dd;
                sq = fma(dd.x, dd.x, fma(dd.y, dd.y, sq));
                if (a.rpart) {
                    const CT r = csub(a.y[i], v);
                    rq = fma(r.x, r.x, fma(r.y, r.y, rq));
                }
            }
        }
    }
    if (MODE == DOUT_PD) {
        const double tot = block_sum((double)sq, red);
        if (threadIdx.x == 0) a.part[it.slot] = tot;
        if (a.rpart) {
            const double rt = block_sum((double)rq, red);
            if (threadIdx.x == 0) a.rpart[it.slot] = rt;
        }
    }
}

// ---------------------------------------------------------------- gridding
// Work item of the gridding kernel: one (channel, tile) list range. Tiles whose
// list is longer than GRID_CAP entries are split into several items; each
// writes its partial tile to a slot of the partial buffer and k_grid_merge
// adds the slots of a tile in a fixed order. Unsplit tiles (slot < 0) write
// the grid directly.
struct GridItem {
    int tix;      // l * ntiles + tile
    int e0, e1;   // entry range in tile_ent
    int slot;     // partial slot, or -1
};

template <typename R, int NC, int MODE, bool KAHAN>
__global__ void __launch_bounds__(GRID_WARPS * 32) k_grid(NufftK<R> a, const GridItem* __restrict__ items,
                                                         Cx<R>* __restrict__ partial) {
    typedef Cx<R> CT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int TX = a.g.tx, TY = a.g.ty;
    const int cells = TX * TY;
    CT* acc = reinterpret_cast<CT*>(smem_raw);             // [GRID_WARPS][cells]
    CT* cmp = acc + (size_t)GRID_WARPS * cells;            // [GRID_WARPS][cells] (KAHAN)
    __shared__ int2 s_k0[GRID_WARPS][32];                  // window start cells of a batch
    __shared__ CT s_val[GRID_WARPS][32];                   // weighted values of a batch
    __shared__ R s_phi[GRID_WARPS][32][17];                // 8 x-taps, 8 y-taps per entry
    const GridItem it = items[blockIdx.x];
    const int ntiles = a.g.ntx * a.g.nty;
    const int l = it.tix / ntiles;
    const int t = it.tix - l * ntiles;
    const int tyi = t / a.g.ntx, txi = t - tyi * a.g.ntx;
    const int ty0 = tyi * TY, tx0 = txi * TX;
    const int Kx = a.g.Kx, Ky = a.g.Ky;
    const int kxm = a.g.kxm, kym = a.g.kym;
    for (int k = threadIdx.x; k < GRID_WARPS * cells; k += blockDim.x) {
        acc[k] = cx<R>(0, 0);
        if (KAHAN) cmp[k] = cx<R>(0, 0);
    }
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int half = lane >> 4, sub = lane & 15;
    R c[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) c[k] = a.kbc[(7 - (sub & 7)) * NC + k];
    CT* mine = acc + (size_t)w * cells;
    CT* mcmp = cmp + (size_t)w * cells;
    const int cc = lane & 7, r0 = lane >> 3;
    // Batches of 32 entries per warp. (1) lane q fetches entry base + q: index,
    // coordinates, weighted value (all loads of the batch in flight together);
    // (2) the 16 kernel taps of every entry are evaluated two entries at a time
    // (16 lanes each) into shared memory; (3) the windows are added one at a time
    // into the warp's private tile, 32 lanes covering 8 columns x 2 x 4 rows.
    for (int base = it.e0 + 32 * w; base < it.e1; base += 32 * GRID_WARPS) {
        const int e = base + lane;
        const int nb = min(32, it.e1 - base);
        R fx = 0, fy = 0;
        const int64_t i = e < it.e1 ? a.tile_ent[e] : -1;   // -1: padding of the plan's groups
        s_k0[w][lane] = make_int2(-1, -1);
        if (i >= 0) {
            int cxv, cyv;
            VisCoord<R>::get(a.coords, i, a.g, cxv, cyv, fx, fy);
            const int k0x = wrapn(cxv - 3, Kx, kxm);
            const int k0y = wrapn(cyv - 3, Ky, kym);
            CT val;
            if (MODE == GIN_CALLER) {
                val = a.in[a.perm[i]];
            } else if (MODE == GIN_SORTED) {
                val = a.in[i];
            } else {   // GIN_PD: v = U^{1/2} d max(0, 1 - eps / rho); the home tile stores it
                val = cscale(a.d[i], a.scale[a.blk ? a.blk[i] : l]);
                if (a.u) val = cscale(val, sqrt(a.u[i]));
                if ((k0x / TX == txi) && (k0y / TY == tyi)) a.v[i] = val;
            }
            if (a.w) val = cscale(val, a.w[i]);
            s_k0[w][lane] = make_int2(k0x, k0y);
            s_val[w][lane] = val;
        }
        for (int k = 0; k < nb; k += 2) {
            const int src = k + half;
            const R fxs = __shfl_sync(0xffffffffu, fx, src);
            const R fys = __shfl_sync(0xffffffffu, fy, src);
            const R phi = horner<R, NC>(c, (R)2 * (sub < 8 ? fxs : fys) - (R)1);
            s_phi[w][src][sub] = phi;
        }
        __syncwarp();
        for (int k = 0; k < nb; ++k) {
            const int2 b0 = s_k0[w][k];
            if (b0.x < 0) continue;
            const int gx = (wrapn(b0.x + cc, Kx, kxm)) - tx0;
            if (gx >= 0 && gx < TX) {
                const CT vv = s_val[w][k];
                const R pu = s_phi[w][k][cc];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int rr = r0 + 4 * q;
                    const int gy = (wrapn(b0.y + rr, Ky, kym)) - ty0;
                    if (gy < 0 || gy >= TY) continue;
                    const R wgt = pu * s_phi[w][k][8 + rr];
                    const int cell = gy * TX + gx;
                    if (KAHAN) {
                        CT sm = mine[cell], kk = mcmp[cell];
                        const R yr = fma(wgt, vv.x, -kk.x), yi = fma(wgt, vv.y, -kk.y);
                        const R tr = sm.x + yr, ti = sm.y + yi;
                        kk.x = (tr - sm.x) - yr;
                        kk.y = (ti - sm.y) - yi;
                        sm.x = tr;
                        sm.y = ti;
                        mine[cell] = sm;
                        mcmp[cell] = kk;
                    } else {
                        CT sm = mine[cell];
                        sm.x = fma(wgt, vv.x, sm.x);
                        sm.y = fma(wgt, vv.y, sm.y);
                        mine[cell] = sm;
                    }
                }
            }
        }
        __syncwarp();
    }
    __syncthreads();
    CT* Gout;
    int64_t gstride;
    if (it.slot < 0) {
        Gout = a.grid_out + (int64_t)l * Ky * Kx + (int64_t)ty0 * Kx + tx0;
        gstride = Kx;
    } else {
        Gout = partial + (int64_t)it.slot * cells;
        gstride = TX;
    }
    for (int k = threadIdx.x; k < cells; k += blockDim.x) {
        CT s = acc[k];
        if (KAHAN) {
            // compensated combine of the per-warp (sum - compensation) values
            R sr = s.x, si = s.y, er = -cmp[k].x, ei = -cmp[k].y;
#pragma unroll
            for (int ww = 1; ww < GRID_WARPS; ++ww) {
                const CT x = acc[(size_t)ww * cells + k];
                const CT y = cmp[(size_t)ww * cells + k];
                R tr = sr + x.x;
                er += (sr - tr) + x.x - y.x;
                sr = tr;
                R ti = si + x.y;
                ei += (si - ti) + x.y - y.y;
                si = ti;
            }
            s.x = sr + er;
            s.y = si + ei;
        } else {
#pragma unroll
            for (int ww = 1; ww < GRID_WARPS; ++ww) s = cadd(s, acc[(size_t)ww * cells + k]);
        }
        const int gy = k / TX, gx = k - gy * TX;
        Gout[(int64_t)gy * gstride + gx] = s;
    }
}

// Gridding kernel for grids smaller than 64 x 64 cells (the sweep needs
// strips that no window reaches twice). The plan orders every tile list in groups of 4
// entries whose windows do not overlap (padding -1). Each of the GRID_PW warps
// of a CTA owns a private copy of the tile in shared memory and adds one group
// per pass: 8 lanes per window (lane j: column j, all 8 rows; the row weights
// are exchanged by shuffles inside the 8 lanes), so the 32 lanes of a pass
// update 4 x 8 distinct cells with plain loads and stores and no atomics. A
// warp fetches the entries of 4 groups at once (one lane per entry) so their
// loads are in flight together. The copies are summed in a fixed order: the
// result is deterministic.
constexpr int GRID_PW = 4;          // warps (private tiles) per CTA
constexpr int GRID_LDT = GRID_TILE + 1;

template <typename R, int NC, int MODE>
__global__ void __launch_bounds__(GRID_PW * 32) k_grid_groups(NufftK<R> a, const GridItem* __restrict__ items,
                                                              Cx<R>* __restrict__ partial) {
    typedef Cx<R> CT;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    CT* priv = reinterpret_cast<CT*>(smem_raw);   // [GRID_PW][GRID_TILE][GRID_LDT]
    constexpr int TCELLS = GRID_TILE * GRID_LDT;
    const GridItem it = items[blockIdx.x];
    const int TX = a.g.tx, TY = a.g.ty;
    const int ntiles = a.g.ntx * a.g.nty;
    const int l = it.tix / ntiles;
    const int t = it.tix - l * ntiles;
    const int tyi = t / a.g.ntx, txi = t - tyi * a.g.ntx;
    const int ty0 = tyi * TY, tx0 = txi * TX;
    const int Kx = a.g.Kx, Ky = a.g.Ky;
    const int kxm = a.g.kxm, kym = a.g.kym;
    for (int k = threadIdx.x; k < GRID_PW * TCELLS; k += blockDim.x) priv[k] = cx<R>(0, 0);
    __syncthreads();
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int j = lane & 7, grp = lane >> 3;
    const unsigned gmask = 0xffu << (8 * grp);
    CT* mine = priv + w * TCELLS;
    R c[NC];
#pragma unroll
    for (int k = 0; k < NC; ++k) c[k] = a.kbc[(7 - j) * NC + k];
    const int ng = (it.e1 - it.e0) >> 2;
    for (int g0 = 4 * w; g0 < ng; g0 += 4 * GRID_PW) {
        const int nbg = min(4, ng - g0);
        // lane 4p + s fetches slot s of group g0 + p
        int k0x = -1, k0y = 0;
        R fx = 0, fy = 0;
        CT val = cx<R>(0, 0);
        if (lane < 4 * nbg) {
            const int64_t i = a.tile_ent[it.e0 + 4 * g0 + lane];
            if (i >= 0) {
                int cxv, cyv;
                VisCoord<R>::get(a.coords, i, a.g, cxv, cyv, fx, fy);
                k0x = wrapn(cxv - 3, Kx, kxm);
                k0y = wrapn(cyv - 3, Ky, kym);
                if (MODE == GIN_CALLER) {
                    val = a.in[a.perm[i]];
                } else if (MODE == GIN_SORTED) {
                    val = a.in[i];
                } else {   // GIN_PD: v = U^{1/2} d max(0, 1 - eps / rho); the home tile stores it
                    val = cscale(a.d[i], a.scale[a.blk ? a.blk[i] : l]);
                    if (a.u) val = cscale(val, sqrt(a.u[i]));
                    if ((k0x / TX == txi) && (k0y / TY == tyi)) a.v[i] = val;
                }
                if (a.w) val = cscale(val, a.w[i]);
            }
        }
        for (int p = 0; p < nbg; ++p) {
            const int src = 4 * p + grp;
            const int sx = __shfl_sync(0xffffffffu, k0x, src);
            const int sy = __shfl_sync(0xffffffffu, k0y, src);
            const R sfx = __shfl_sync(0xffffffffu, fx, src);
            const R sfy = __shfl_sync(0xffffffffu, fy, src);
            const R vr = __shfl_sync(0xffffffffu, val.x, src);
            const R vi = __shfl_sync(0xffffffffu, val.y, src);
            if (sx < 0) continue;   // padding; uniform over the 8 lanes of a window
            const R phx = horner<R, NC>(c, (R)2 * sfx - (R)1);   // phi_u of column j
            const R phy = horner<R, NC>(c, (R)2 * sfy - (R)1);   // phi_v of row j
            const int gx = (wrapn(sx + j, Kx, kxm)) - tx0;
            const bool colok = (unsigned)gx < (unsigned)TX;
            const R pr = phx * vr, pi = phx * vi;
            // the 8 rows of a window are distinct cells: load all, add, store all
            CT cur[8];
            int off[8];
            bool ok[8];
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const int gy = (wrapn(sy + r, Ky, kym)) - ty0;
                ok[r] = colok && (unsigned)gy < (unsigned)TY;
                off[r] = gy * GRID_LDT + gx;
                if (ok[r]) cur[r] = mine[off[r]];
            }
#pragma unroll
            for (int r = 0; r < 8; ++r) {
                const R pw = __shfl_sync(gmask, phy, r, 8);
                if (ok[r]) {
                    cur[r].x = fma(pw, pr, cur[r].x);
                    cur[r].y = fma(pw, pi, cur[r].y);
                    mine[off[r]] = cur[r];
                }
            }
        }
    }
    __syncthreads();
    CT* Gout;
    int64_t gstride;
    if (it.slot < 0) {
        Gout = a.grid_out + (int64_t)l * Ky * Kx + (int64_t)ty0 * Kx + tx0;
        gstride = Kx;
    } else {
        Gout = partial + (int64_t)it.slot * TX * TY;
        gstride = TX;
    }
    for (int k = threadIdx.x; k < GRID_TILE * GRID_TILE; k += blockDim.x) {
        const int gy = k >> 5, gx = k & (GRID_TILE - 1);
        if (gy < TY && gx < TX) {
            CT s = priv[gy * GRID_LDT + gx];
#pragma unroll
            for (int ww = 1; ww < GRID_PW; ++ww) s = cadd(s, priv[ww * TCELLS + gy * GRID_LDT + gx]);
            Gout[(int64_t)gy * gstride + gx] = s;
        }
    }
}

// Sweep gridding (grids of at least 64 x 64 cells, default kernel). A warp owns
// one work item of the plan: a 32-column strip of one channel's grid and its
// output rows [row0, row1). Lane c holds column c of three 4-row register
// banks; band j (rows 4j .. 4j + 3 relative to row0) lives in bank j mod 3. The
// warp walks the item's groups band by band: a group holds up to 4 windows with
// disjoint columns starting in band j, so they lie in bands j .. j + 2 and one
// pass over those 12 rows (2 x 12 FMAs per lane) adds them; once a group of a
// later band arrives, band j is final, so its bank is stored (each output cell
// once, coalesced 256-byte rows) and cleared for band j + 3. The banks never
// move between registers, there is no shared-memory read-modify-write, no
// atomics, and the summation order is fixed.
// Lists are consumed in batches of 32 slots (8 groups): lane q decodes slot q
// (window position, weighted value, the 16 kernel taps) into shared memory: the
// 8 row taps at their rows of the 12-row span (zeros elsewhere), and for
// every strip column the window covers, the column tap times the value and the
// slot's place in its group, tagged with the batch number (a column whose entry
// carries an older tag has no window in the group and adds zero, so the table
// is never cleared), and the group pass reads one 8-byte value and one 4-byte
// tag per lane. The
// next batch's list entries and inputs are loaded before the current batch's
// groups are added.
constexpr int SW_WARPS = 4;      // warps (work items) per CTA

// 4 consecutive reals from 16-byte aligned shared memory
__device__ __forceinline__ void sw_ld4(const float* p, float* v) {
    const float4 t = *reinterpret_cast<const float4*>(p);
    v[0] = t.x; v[1] = t.y; v[2] = t.z; v[3] = t.w;
}
__device__ __forceinline__ void sw_ld4(const double* p, double* v) {
    const double2 t0 = reinterpret_cast<const double2*>(p)[0], t1 = reinterpret_cast<const double2*>(p)[1];
    v[0] = t0.x; v[1] = t0.y; v[2] = t1.x; v[3] = t1.y;
}

// Inputs of one list slot loaded ahead of its decoding.
template <typename R> struct SwRaw {
    typename CxT<R>::T v;   // value (GIN_SORTED), d (GIN_PD)
    R u, w;                 // U and Theta of the visibility (1 when absent)
    int p;                  // caller index (GIN_CALLER) or data block (GIN_PD with blocks)
};

template <typename R, int NC, int MODE>
__global__ void __launch_bounds__(SW_WARPS * 32, sizeof(R) == 4 ? 5 : 1)
    k_grid_sweep(const NufftK<R> a, const SweepItem* __restrict__ items,
                 const int* __restrict__ ent, int n_items) {
    typedef Cx<R> CT;
    constexpr int NE = (NC + 1) / 2, NO = NC / 2;   // even / odd coefficients of a piece
    // row taps of every slot, placed at their rows; with 12 reals per slot the 4
    // slots of a group fall in disjoint banks for 16-byte loads
    constexpr int RLD = 12;
    __shared__ __align__(16) R rowt[SW_WARPS][32][RLD];
    // per group and strip column: column tap x value, and 4 x batch + slot in the
    // group (rows padded to 33 entries: the decode's scattered stores of different
    // groups fall in different banks)
    __shared__ __align__(16) CT coltv[SW_WARPS][8][33];
    __shared__ int coltg[SW_WARPS][8][33];
    __shared__ int sjb[SW_WARPS][8];                          // band of every group
    const int w = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int wi = blockIdx.x * SW_WARPS + w;
    if (wi >= n_items) return;
    const SweepItem it = items[wi];
    const int Kx = a.g.Kx, Ky = a.g.Ky;
    const int kxm = a.g.kxm, kym = a.g.kym;
    const int c0 = it.strip * GRID_TILE, row0 = it.row0, H = it.row1 - it.row0;
    CT* out = a.grid_out + (int64_t)it.l * Ky * Kx + (int64_t)row0 * Kx + c0 + lane;
    CT B0[4], B1[4], B2[4];
#pragma unroll
    for (int k = 0; k < 4; ++k) B0[k] = B1[k] = B2[k] = cx<R>(0, 0);
    int jb = -2;   // band whose rows are final next (rows -8 .. -1 are never stored)
    int jm = 1;    // its bank, jb mod 3

    // ---- loads of one slot's inputs (list entry i, -1 = padding)
    auto load_raw = [&](int i, SwRaw<R>& r) {
        r.u = r.w = (R)1;
        r.p = 0;
        if (i < 0) return;
        if (MODE == GIN_CALLER) {
            r.p = a.perm[i];
        } else if (MODE == GIN_SORTED) {
            r.v = reinterpret_cast<const typename CxT<R>::T*>(a.in)[i];
        } else {
            r.v = reinterpret_cast<const typename CxT<R>::T*>(a.d)[i];
            if (a.blk) r.p = a.blk[i];
            if (a.u) r.u = a.u[i];
        }
        if (a.w) r.w = a.w[i];
    };
    // ---- kernel taps of one axis: tap m is piece 7 - m of the window at s; pieces
    // 7 - m and m are mirror images (phi is even), so taps m and 7 - m are
    // E(s^2) + s O(s^2) and E(s^2) - s O(s^2) of piece 7 - m
    auto taps = [&](R s, R* t) {
        const R s2 = s * s;
#pragma unroll
        for (int m = 0; m < 4; ++m) {
            R e = a.kev[m * KB_HALF + NE - 1];
#pragma unroll
            for (int k = NE - 2; k >= 0; --k) e = fma(e, s2, a.kev[m * KB_HALF + k]);
            R o = a.kod[m * KB_HALF + NO - 1];
#pragma unroll
            for (int k = NO - 2; k >= 0; --k) o = fma(o, s2, a.kod[m * KB_HALF + k]);
            t[m] = fma(s, o, e);
            t[7 - m] = fma(-s, o, e);
        }
    };
    // ---- store the final band jb (rows 8 jb .. 8 jb + 7 inside [0, H)) and clear its bank
    auto flush = [&](CT(&U)[4]) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            const int r = 4 * jb + k;
            if ((unsigned)r < (unsigned)H) out[(int64_t)r * Kx] = U[k];
            U[k] = cx<R>(0, 0);
        }
    };
    auto advance = [&]() {
        if (jm == 0) flush(B0);
        else if (jm == 1) flush(B1);
        else flush(B2);
        ++jb;
        jm = jm == 2 ? 0 : jm + 1;
    };
    auto add = [&](CT(&U)[4], CT(&V)[4], CT(&W)[4], const R* pv, CT t) {
#pragma unroll
        for (int k = 0; k < 4; ++k) {
            U[k].x = fma(pv[k], t.x, U[k].x);
            U[k].y = fma(pv[k], t.y, U[k].y);
            V[k].x = fma(pv[4 + k], t.x, V[k].x);
            V[k].y = fma(pv[4 + k], t.y, V[k].y);
            W[k].x = fma(pv[8 + k], t.x, W[k].x);
            W[k].y = fma(pv[8 + k], t.y, W[k].y);
        }
    };

    int i_cur = it.e0 + lane < it.e1 ? ent[it.e0 + lane] : -1;
    SwRaw<R> r_cur;
    load_raw(i_cur, r_cur);
    int i_nxt = it.e0 + 32 + lane < it.e1 ? ent[it.e0 + 32 + lane] : -1;
    R* rt = rowt[w][lane];
    for (int k = lane; k < 8 * 33; k += 32) {
        (&coltv[w][0][0])[k] = cx<R>(0, 0);
        (&coltg[w][0][0])[k] = -1;
    }
    __syncwarp();
    int nbat = 0;   // batch number (tag of the column entries written by this batch)
    for (int b0 = it.e0; b0 < it.e1; b0 += 32) {
        // ---- decode slot b0 + lane
        const int i = i_cur;
        const SwRaw<R> r = r_cur;
        i_cur = i_nxt;
        load_raw(i_cur, r_cur);   // next batch's inputs (their entries were loaded a batch ago)
        i_nxt = b0 + 64 + lane < it.e1 ? ent[b0 + 64 + lane] : -1;
        int ry = 0;
        if (i >= 0) {
            int cxv, cyv;
            R fx, fy;
            VisCoord<R>::get(a.coords, i, a.g, cxv, cyv, fx, fy);
            const int k0x = wrapn(cxv - 3, Kx, kxm);
            const int k0y = wrapn(cyv - 3, Ky, kym);
            const int rx = (wrapn(k0x - c0 + 7, Kx, kxm)) - 7;     // -7 .. 31
            ry = (wrapn(k0y - row0 + 7, Ky, kym)) - 7;              // -7 .. H - 1
            CT val;
            if (MODE == GIN_CALLER) {
                val = a.in[r.p];
            } else if (MODE == GIN_SORTED) {
                val = cx<R>(r.v.x, r.v.y);
            } else {   // GIN_PD: v = U^{1/2} d max(0, 1 - eps / rho); the item holding the window start stores it
                val = cscale(cx<R>(r.v.x, r.v.y), a.scale[a.blk ? r.p : it.l]);
                if (a.u) val = cscale(val, sqrt(r.u));
                if (rx >= 0 && ry >= 0 && ry < H) a.v[i] = val;
            }
            if (a.w) val = cscale(val, r.w);
            R pu[8], pv[8];
            taps((R)2 * fx - (R)1, pu);   // phi_u of window columns 0 .. 7
            taps((R)2 * fy - (R)1, pv);   // phi_v of window rows 0 .. 7
#pragma unroll
            for (int k = 0; k < 3 * (int)sizeof(R) / 4; ++k)   // 12 reals
                reinterpret_cast<float4*>(rt)[k] = make_float4(0.f, 0.f, 0.f, 0.f);
            R* sr = rt + (ry & 3);   // row m of the window is row (ry & 3) + m of the three bands
#pragma unroll
            for (int m = 0; m < 8; ++m) sr[m] = pv[m];
            const int g = lane >> 2;
#pragma unroll
            for (int m = 0; m < 8; ++m) {
                const int c = rx + m;
                if ((unsigned)c < 32u)
                {
                    coltv[w][g][c] = cx<R>(pu[m] * val.x, pu[m] * val.y);
                    coltg[w][g][c] = (nbat << 2) | (lane & 3);
                }
            }
        }
        if ((lane & 3) == 0) sjb[w][lane >> 2] = ry >> 2;
        __syncwarp();
        // ---- add the batch's groups
        // (each group's column entry and band are read one group ahead)
        const int ng = min(8, (it.e1 - b0) >> 2);
        CT cv_n = coltv[w][0][lane];
        int cg_n = coltg[w][0][lane];
        int gj_n = sjb[w][0];
        for (int q = 0; q < ng; ++q) {
            const CT cv = cv_n;
            const int cg = cg_n;
            const int gj = gj_n;
            const bool cur = (cg >> 2) == nbat;
            const R* pvs = rowt[w][4 * q + (cur ? (cg & 3) : 0)];
            R pv[12];
#pragma unroll
            for (int k = 0; k < 12; k += 4) sw_ld4(pvs + k, pv + k);
            const int qn = min(q + 1, 7);
            cv_n = coltv[w][qn][lane];
            cg_n = coltg[w][qn][lane];
            gj_n = sjb[w][qn];
            while (jb < gj) advance();
            const CT t = cur ? cv : cx<R>(0, 0);
            if (jm == 0) add(B0, B1, B2, pv, t);
            else if (jm == 1) add(B1, B2, B0, pv, t);
            else add(B2, B0, B1, pv, t);
        }
        __syncwarp();
        ++nbat;
    }
    while (4 * jb < H) advance();
}

// Sum of the partial tiles of every split tile (fixed slot order).
struct GridMerge {
    int tix, slot0, nslot;
};

template <typename R>
__global__ void k_grid_merge(const GridMerge* __restrict__ merges, const Cx<R>* __restrict__ partial,
                             Cx<R>* __restrict__ grid, Geo g) {
    typedef Cx<R> CT;
    const GridMerge m = merges[blockIdx.x];
    const int cells = g.tx * g.ty;
    const int ntiles = g.ntx * g.nty;
    const int l = m.tix / ntiles, t = m.tix - l * ntiles;
    const int tyi = t / g.ntx, txi = t - tyi * g.ntx;
    CT* G = grid + (int64_t)l * g.Ky * g.Kx + (int64_t)(tyi * g.ty) * g.Kx + txi * g.tx;
    for (int k = threadIdx.x; k < cells; k += blockDim.x) {
        CT s = partial[(int64_t)m.slot0 * cells + k];
        for (int j = 1; j < m.nslot; ++j) s = cadd(s, partial[(int64_t)(m.slot0 + j) * cells + k]);
        const int gy = k / g.tx, gx = k - gy * g.tx;
        G[(int64_t)gy * g.Kx + gx] = s;
    }
}

// ---------------------------------------------------------------- launches
int degrid_blocks_x(const Plan* p) { return (p->Mmax + DEGRID_CHUNK - 1) / DEGRID_CHUNK; }
int degrid_items_max(const Plan* p) { return p->dg_items_max > 0 ? p->dg_items_max : 1; }

template <typename R> static NufftK<R> base_args(Plan* p) {
    NufftK<R> k{};
    k.g = p->g;
    k.grid = (const Cx<R>*)p->grid;
    k.grid_out = (Cx<R>*)p->grid;
    k.coords = p->coords;
    k.off = p->off_d;
    k.w = (const R*)p->w_sorted;
    k.u = (const R*)p->u_sorted;
    k.perm = p->perm;
    k.kbc = (const R*)p->kbc;
    const int nc = p->kb_terms;
    for (int m = 0; m < 4; ++m)
        for (int j = 0; j < nc; ++j) {
            const R c = (R)p->kbc_h[(size_t)(7 - m) * nc + j];
            if (j & 1) k.kod[m * KB_HALF + j / 2] = c;
            else k.kev[m * KB_HALF + j / 2] = c;
        }
    k.tile_off = p->tile_off;
    k.tile_ent = p->tile_ent;
    k.blk = p->blk_id;
    k.nblk_x = degrid_blocks_x(p);
    return k;
}

template <typename R, int NC>
static hs_status degrid_t(Plan* p, const DegridArgs& da, cudaStream_t s) {
    NufftK<R> k = base_args<R>(p);
    k.out = (Cx<R>*)da.out;
    k.v = (Cx<R>*)da.v;
    k.y = (const Cx<R>*)da.y;
    k.d = (Cx<R>*)da.d;
    k.part = da.part;
    k.rpart = da.rpart;
    if (p->n_dg_items == 0) return HS_OK;
    const unsigned nb = (unsigned)p->n_dg_items;
    const size_t sm = (size_t)DG_REG * DG_LDS * sizeof(Cx<R>);
    const DgItem* items = (const DgItem*)p->dg_items;
    switch (da.mode) {
        case DOUT_CALLER: k_degrid<R, NC, DOUT_CALLER><<<nb, 256, sm, s>>>(k, items); break;
        case DOUT_SORTED: k_degrid<R, NC, DOUT_SORTED><<<nb, 256, sm, s>>>(k, items); break;
        case DOUT_SORTED_U: k_degrid<R, NC, DOUT_SORTED_U><<<nb, 256, sm, s>>>(k, items); break;
        case DOUT_PD: k_degrid<R, NC, DOUT_PD><<<nb, 256, sm, s>>>(k, items); break;
        default: return fail(HS_ERR_ARG, "degrid: bad mode");
    }
    HS_CHECK_LAUNCH();
    return HS_OK;
}

hs_status degrid(Plan* p, const DegridArgs& a, cudaStream_t s) {
    if (p->prec == HS_F32) return degrid_t<float, KB_TERMS_F32>(p, a, s);
    return degrid_t<double, KB_TERMS_F64>(p, a, s);
}

template <typename R, int NC, int MODE, bool KAHAN>
static hs_status grid_launch(Plan* p, NufftK<R>& k, cudaStream_t s) {
    const size_t smem = (size_t)GRID_WARPS * p->g.tx * p->g.ty * sizeof(Cx<R>) * (KAHAN ? 2 : 1);
    if (!KAHAN && p->n_sw_items > 0) {
        const unsigned nb = (unsigned)((p->n_sw_items + SW_WARPS - 1) / SW_WARPS);
        k_grid_sweep<R, NC, MODE><<<nb, SW_WARPS * 32, 0, s>>>(k, (const SweepItem*)p->sw_items, p->sw_ent,
                                                             (int)p->n_sw_items);
        HS_CHECK_LAUNCH();
        return HS_OK;
    }
    if (p->n_items == 0) return HS_OK;
    if (KAHAN)
        k_grid<R, NC, MODE, KAHAN><<<(unsigned)p->n_items, GRID_WARPS * 32, smem, s>>>(
            k, (const GridItem*)p->grid_items, (Cx<R>*)p->grid_partial);
    else
        k_grid_groups<R, NC, MODE><<<(unsigned)p->n_items, GRID_PW * 32,
                                     (size_t)GRID_PW * GRID_TILE * GRID_LDT * sizeof(Cx<R>), s>>>(
            k, (const GridItem*)p->grid_items, (Cx<R>*)p->grid_partial);
    HS_CHECK_LAUNCH();
    if (p->n_merges > 0) {
        k_grid_merge<R><<<(unsigned)p->n_merges, 256, 0, s>>>((const GridMerge*)p->grid_merges,
                                                            (const Cx<R>*)p->grid_partial,
                                                            (Cx<R>*)p->grid, p->g);
        HS_CHECK_LAUNCH();
    }
    return HS_OK;
}

template <typename R, int NC, int MODE, bool KAHAN> static hs_status grid_attr() {
    const int smem = GRID_WARPS * GRID_TILE * GRID_TILE * (int)sizeof(Cx<R>) * (KAHAN ? 2 : 1);
    static_assert(sizeof(GridItem) == 16 && sizeof(GridMerge) == 12, "plan-side layout");
    HS_CHECK_CUDA(cudaFuncSetAttribute(k_grid<R, NC, MODE, KAHAN>,
                                       cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    if (!KAHAN)
        HS_CHECK_CUDA(cudaFuncSetAttribute(k_grid_groups<R, NC, MODE>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                           (int)(GRID_PW * GRID_TILE * GRID_LDT * sizeof(Cx<R>))));
    return HS_OK;
}

// Opt the gridding kernels into their dynamic shared memory (once per process).
hs_status nufft_init() {
    static bool done = false;
    if (done) return HS_OK;
    HS_TRY((grid_attr<float, KB_TERMS_F32, GIN_CALLER, false>()));
    HS_TRY((grid_attr<float, KB_TERMS_F32, GIN_SORTED, false>()));
    HS_TRY((grid_attr<float, KB_TERMS_F32, GIN_PD, false>()));
    HS_TRY((grid_attr<float, KB_TERMS_F32, GIN_CALLER, true>()));
    HS_TRY((grid_attr<float, KB_TERMS_F32, GIN_SORTED, true>()));
    HS_TRY((grid_attr<float, KB_TERMS_F32, GIN_PD, true>()));
    HS_TRY((grid_attr<double, KB_TERMS_F64, GIN_CALLER, false>()));
    HS_TRY((grid_attr<double, KB_TERMS_F64, GIN_SORTED, false>()));
    HS_TRY((grid_attr<double, KB_TERMS_F64, GIN_PD, false>()));
    HS_TRY((grid_attr<double, KB_TERMS_F64, GIN_CALLER, true>()));
    HS_TRY((grid_attr<double, KB_TERMS_F64, GIN_SORTED, true>()));
    HS_TRY((grid_attr<double, KB_TERMS_F64, GIN_PD, true>()));
    done = true;
    return HS_OK;
}

template <typename R, int NC, bool KAHAN>
static hs_status grid_t(Plan* p, const GridArgs& ga, cudaStream_t s) {
    NufftK<R> k = base_args<R>(p);
    k.in = (const Cx<R>*)ga.in;
    k.d = (Cx<R>*)ga.d;
    k.scale = (const R*)ga.scale;
    k.v = (Cx<R>*)ga.v;
    if (p->g.L == 0) return HS_OK;
    switch (ga.mode) {
        case GIN_CALLER: return grid_launch<R, NC, GIN_CALLER, KAHAN>(p, k, s);
        case GIN_SORTED: return grid_launch<R, NC, GIN_SORTED, KAHAN>(p, k, s);
        case GIN_PD: return grid_launch<R, NC, GIN_PD, KAHAN>(p, k, s);
        default: return fail(HS_ERR_ARG, "grid: bad mode");
    }
}

hs_status grid(Plan* p, const GridArgs& a, cudaStream_t s) {
    if (p->prec == HS_F32) {
        if (p->flags & HS_PLAN_COMPENSATED) return grid_t<float, KB_TERMS_F32, true>(p, a, s);
        return grid_t<float, KB_TERMS_F32, false>(p, a, s);
    }
    if (p->flags & HS_PLAN_COMPENSATED) return grid_t<double, KB_TERMS_F64, true>(p, a, s);
    return grid_t<double, KB_TERMS_F64, false>(p, a, s);
}

}  // namespace hs
