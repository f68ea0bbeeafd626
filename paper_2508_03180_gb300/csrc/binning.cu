// Cell rasterization (Layer I, Sec. IV-B): project every ellipsoidal cell
// proxy of every view, cull it to the frustum, bound its screen footprint,
// and emit one (tile, cell) pair per covered tile.  Depth ordering comes from
// a radix sort over cells (sort.cu); a second stable sort groups by tile.
#include "internal.cuh"
#include "sh.cuh"

namespace dgs {

// One thread per (view, cell).  Footprint: exact screen bounding box of the
// perspective image of the ellipsoid {c + R_Q diag(S) u, |u| <= 1}.  With the
// view-space centre c and Sigma = M M^T (M = R_view R_Q diag(S)) the planes
// X - t Z = 0 tangent to the ellipsoid solve
//   (c_z^2 - S_zz) t^2 - 2 (c_x c_z - S_xz) t + (c_x^2 - S_xx) = 0,
// whose discriminant is expanded so the c_x^2 c_z^2 terms cancel exactly.
// All of it in FP32 with a fixed operation order (see internal.cuh), so the
// tile rectangle is reproducible bit for bit.
__global__ void __launch_bounds__(256) k_cell_project(const ViewDesc *__restrict__ views, int n_views,
                                                      const SceneDev *__restrict__ scenes,
                                                      uint32_t *__restrict__ zkey, uint32_t *__restrict__ zval,
                                                      short4 *__restrict__ rect, float *__restrict__ depth,
                                                      uint32_t *__restrict__ count, uint32_t *__restrict__ visible,
                                                      float *__restrict__ vview, int flags,
                                                      const ChainSizes *__restrict__ dsz) {
    if (dsz) n_views = dsz->n_views;
    uint32_t nvis = 0;
    for (int v = 0; v < n_views; ++v) {
    const ViewDesc &V = views[v];
    const SceneDev &SC = scenes[V.scene_slot];
    const float *__restrict__ cell = SC.cell;
    const long long N = V.N;
    for (long long n = blockIdx.x * (long long)blockDim.x + threadIdx.x; n < N;
         n += (long long)gridDim.x * blockDim.x) {
        const long long i = V.cell_base + n;
        float c[3];
        xform_s(V.R, V.t, cell[n], cell[N + n], cell[2 * N + n], c);
        float Rq[9], RR[9], M[9];
        rot_from_quat_s(cell[6 * N + n], cell[7 * N + n], cell[8 * N + n], cell[9 * N + n], Rq);
        const float S[3] = {cell[3 * N + n], cell[4 * N + n], cell[5 * N + n]};
#pragma unroll
        for (int a = 0; a < 3; ++a)
#pragma unroll
            for (int j = 0; j < 3; ++j) {
                RR[3 * a + j] = fadd_s(fadd_s(fmul_s(V.R[3 * a], Rq[j]), fmul_s(V.R[3 * a + 1], Rq[3 + j])),
                                       fmul_s(V.R[3 * a + 2], Rq[6 + j]));
                M[3 * a + j] = fmul_s(RR[3 * a + j], S[j]);
            }
        auto sig = [&](int a, int b) {
            return fadd_s(fadd_s(fmul_s(M[3 * a], M[3 * b]), fmul_s(M[3 * a + 1], M[3 * b + 1])),
                          fmul_s(M[3 * a + 2], M[3 * b + 2]));
        };
        const float sxx = sig(0, 0), syy = sig(1, 1), szz = sig(2, 2), sxz = sig(0, 2), syz = sig(1, 2);
        float dz = c[2];  // the sort depth
        short4 r = make_short4(-1, -1, -1, -1);
        bool vis = fsub_s(c[2], fsqrt_s(szz)) > V.znear;
        if (!vis && (flags & DGS_FLAG_NEAR_FULL) && fadd_s(c[2], fsqrt_s(szz)) > V.znear) {
            // straddles the near plane: conservatively every tile, nearest first
            vis = true;
            dz = c[2] > 0.0f ? c[2] : 0.0f;
            r = make_short4(0, 0, (short)(V.Tx - 1), (short)(V.Ty - 1));
        } else if (vis) {
            const float czz = fmul_s(c[2], c[2]);
            const float a = fsub_s(czz, szz);
            float lo[2], hi[2];
#pragma unroll
            for (int ax = 0; ax < 2; ++ax) {
                const float cu = c[ax];
                const float suu = ax == 0 ? sxx : syy, suz = ax == 0 ? sxz : syz;
                const float f = ax == 0 ? V.fx : V.fy, pp = ax == 0 ? V.cx : V.cy;
                const float cuz = fmul_s(cu, c[2]), cuu = fmul_s(cu, cu);
                const float b = fsub_s(cuz, suz);
                float disc = fsub_s(fadd_s(fsub_s(fmul_s(czz, suu), fmul_s(fmul_s(2.0f, cuz), suz)), fmul_s(cuu, szz)),
                                    fsub_s(fmul_s(suu, szz), fmul_s(suz, suz)));
                disc = fmaxf(disc, 0.0f);
                const float sq = fsqrt_s(disc);
                lo[ax] = fadd_s(fmul_s(f, fdiv_s(fsub_s(b, sq), a)), pp);
                hi[ax] = fadd_s(fmul_s(f, fdiv_s(fadd_s(b, sq), a)), pp);
            }
            const float fW = (float)V.W, fH = (float)V.H;
            vis = hi[0] >= 0.0f && lo[0] < fW && hi[1] >= 0.0f && lo[1] < fH;
            if (vis) {
                const float ft = (float)kTile;
                int tx0 = (int)floorf(fdiv_s(fmaxf(lo[0], 0.0f), ft));
                int ty0 = (int)floorf(fdiv_s(fmaxf(lo[1], 0.0f), ft));
                int tx1 = (int)floorf(fdiv_s(fminf(hi[0], fW), ft));
                int ty1 = (int)floorf(fdiv_s(fminf(hi[1], fH), ft));
                tx1 = min(tx1, V.Tx - 1);
                ty1 = min(ty1, V.Ty - 1);
                r = make_short4((short)tx0, (short)ty0, (short)tx1, (short)ty1);
            }
        }
        rect[i] = r;
        depth[i] = dz;
        // v_n of this view (Sec. V-A): the scalar, or clamp(sum_lm k_lm Y_lm(d), 0, 1)
        // with d the unit vector from the eye to the cell centre
        float vn = cell[10 * N + n];
        if (SC.vsh) {
            float d0 = cell[n] - V.eye[0], d1 = cell[N + n] - V.eye[1], d2 = cell[2 * N + n] - V.eye[2];
            const float il = rsqrtf(d0 * d0 + d1 * d1 + d2 * d2);
            d0 *= il; d1 *= il; d2 *= il;
            float Y[16];
            sh_eval(d0, d1, d2, SC.v_sh_degree, Y);
            const int Cv = (SC.v_sh_degree + 1) * (SC.v_sh_degree + 1);
            float raw = 0.f;
            for (int c = 0; c < Cv; ++c) raw += SC.vsh[c * N + n] * Y[c];
            vn = fminf(fmaxf(raw, 0.f), 1.f);
        }
        vview[i] = vn;
        // depth key: positive float bits order like the floats; culled last
        zkey[i] = vis ? __float_as_uint(dz) : 0xFFFFFFFFu;
        zval[i] = (uint32_t)i;
        count[i] = vis ? (uint32_t)((r.z - r.x + 1) * (r.w - r.y + 1)) : 0u;
        nvis += vis ? 1u : 0u;
    }
    }
    // one atomic per warp for the visible-cell statistic
#pragma unroll
    for (int o = 16; o > 0; o >>= 1) nvis += __shfl_xor_sync(0xffffffffu, nvis, o);
    if ((threadIdx.x & 31) == 0 && nvis) atomicAdd(visible, nvis);
}

static int grid_for(long long n, int threads) {
    long long b = (n + threads - 1) / threads;
    const long long cap = 152LL * 32;  // 152 SMs x resident blocks; grid-stride beyond
    if (b > cap) b = cap;
    return (int)(b < 1 ? 1 : b);
}

void launch_cell_project(const ViewDesc *views, int n_views, const SceneDev *scenes, long long n_entries,
                         uint32_t *zkey, uint32_t *zval, short4 *rect, float *depth, uint32_t *count,
                         uint32_t *visible, float *vview, int flags, cudaStream_t st, const ChainSizes *dsz) {
    if (n_entries == 0) return;
    k_cell_project<<<grid_for(n_entries / n_views + 1, 256), 256, 0, st>>>(views, n_views, scenes, zkey, zval, rect,
                                                                          depth, count, visible, vview, flags, dsz);
}

__global__ void k_gather_counts(const uint32_t *__restrict__ idx, const uint32_t *__restrict__ count, long long n,
                                const uint32_t *__restrict__ d_n, uint32_t *__restrict__ out) {
    if (d_n) n = *d_n;
    for (long long i = blockIdx.x * (long long)blockDim.x + threadIdx.x; i < n; i += (long long)gridDim.x * blockDim.x)
        out[i] = count[idx[i]];
}

void launch_gather_counts(const uint32_t *zval_sorted, const uint32_t *count, long long n, uint32_t *out,
                          cudaStream_t st, const uint32_t *d_n) {
    if (n == 0) return;
    k_gather_counts<<<grid_for(n, 256), 256, 0, st>>>(zval_sorted, count, n, d_n, out);
}

// Output slot j belongs to the last entry e with offs[e] <= j.  A block takes
// runs of EM_TB consecutive slots: thread 0 finds the run's first and last
// owners by binary search in global memory; when at most EM_TB entries lie
// between them (always for the depth-sorted cell entries, whose culled ones
// come last, so every entry in a run owns a slot) their offsets are staged
// in shared memory and each thread finds its slots' owners there, otherwise
// (entries that own no slot interleaved, as in the weighted-sum comparator's
// index order) it searches the run's entries in global memory.  Consecutive
// threads write consecutive addresses whatever the footprints.  Entries are in depth order, so the emitted sequence is
// (depth, cell)-ordered within every tile; the stable tile sort keeps that order.
constexpr int EM_THREADS = 256, EM_ITEMS = 8, EM_TB = EM_THREADS * EM_ITEMS;
__global__ void __launch_bounds__(EM_THREADS) k_emit(const uint32_t *__restrict__ offs,
                                                     const uint32_t *__restrict__ zval,
                                                     const short4 *__restrict__ rect,
                                                     const ViewDesc *__restrict__ views, int n_views,
                                                     long long n_entries, long long L, uint32_t *__restrict__ tkey,
                                                     uint32_t *__restrict__ tval,
                                                     const ChainSizes *__restrict__ dsz,
                                                     const uint32_t *__restrict__ d_L) {
    __shared__ uint32_t s_off[EM_TB];
    __shared__ long long s_e0, s_ne;
    if (dsz) {
        n_views = dsz->n_views;
        n_entries = dsz->n_entries;
    }
    if (d_L) L = *d_L;
    for (long long j0 = blockIdx.x * (long long)EM_TB; j0 < L; j0 += (long long)gridDim.x * EM_TB) {
        const long long j1 = min(j0 + (long long)EM_TB, L);  // this run: [j0, j1)
        if (threadIdx.x == 0) {
            auto owner = [&](long long j) {
                long long lo = 0, hi = n_entries;
                while (hi - lo > 1) {
                    const long long mid = (lo + hi) >> 1;
                    if ((long long)offs[mid] <= j) lo = mid; else hi = mid;
                }
                return lo;
            };
            const long long e0 = owner(j0);
            s_e0 = e0;
            s_ne = owner(j1 - 1) - e0 + 1;
        }
        __syncthreads();
        const long long e0 = s_e0, ne = s_ne;  // the run's owners are entries [e0, e0 + ne)
        const bool staged = ne <= EM_TB;
        if (staged)
            for (int i = threadIdx.x; i < (int)ne; i += EM_THREADS) s_off[i] = offs[e0 + i];
        __syncthreads();
#pragma unroll 2
        for (int it = 0; it < EM_ITEMS; ++it) {
            const long long j = j0 + it * EM_THREADS + threadIdx.x;
            if (j >= j1) break;
            long long lo = 0, hi = ne;  // last i in [0, ne) with offs[e0 + i] <= j
            while (hi - lo > 1) {
                const long long mid = (lo + hi) >> 1;
                const uint32_t o = staged ? s_off[mid] : offs[e0 + mid];
                if ((long long)o <= j) lo = mid; else hi = mid;
            }
            const uint32_t base = staged ? s_off[lo] : offs[e0 + lo];
            const uint32_t vi = zval[e0 + lo];
            int vlo = 0, vhi = n_views;  // view owning entry vi
            while (vhi - vlo > 1) {
                const int mid = (vlo + vhi) >> 1;
                if (views[mid].cell_base <= (long long)vi) vlo = mid; else vhi = mid;
            }
            const ViewDesc &V = views[vlo];
            const uint32_t cellid = (uint32_t)((long long)vi - V.cell_base);
            const short4 r = rect[vi];
            const int w = r.z - r.x + 1;
            const int local = (int)(j - base);
            const int ty = r.y + local / w, tx = r.x + local % w;
            tkey[j] = (uint32_t)(V.tile_base + ty * V.Tx + tx);
            tval[j] = cellid;
        }
        __syncthreads();  // s_off is refilled for the next run
    }
}

void launch_emit(const uint32_t *offs, const uint32_t *zval_sorted, const short4 *rect, const ViewDesc *views,
                 int n_views, long long n_entries, long long L, uint32_t *tkey, uint32_t *tval, cudaStream_t st,
                 const ChainSizes *dsz, const uint32_t *d_L) {
    if (L == 0) return;
    k_emit<<<grid_for((L + EM_ITEMS - 1) / EM_ITEMS, EM_THREADS), EM_THREADS, 0, st>>>(
        offs, zval_sorted, rect, views, n_views, n_entries, L, tkey, tval, dsz, d_L);
}

// [start, end) of every non-empty tile from the tile-sorted keys; empty
// tiles keep the (0,0) the caller cleared them to.
__global__ void k_tile_ranges(const uint32_t *__restrict__ key, long long L, const uint32_t *__restrict__ d_L,
                              uint2 *__restrict__ ranges) {
    if (d_L) L = *d_L;
    for (long long j = blockIdx.x * (long long)blockDim.x + threadIdx.x; j < L; j += (long long)gridDim.x * blockDim.x) {
        const uint32_t k = key[j];
        if (j == 0 || key[j - 1] != k) ranges[k].x = (uint32_t)j;
        if (j == L - 1 || key[j + 1] != k) ranges[k].y = (uint32_t)(j + 1);
    }
}

void launch_tile_ranges(const uint32_t *tkey_sorted, long long L, uint2 *ranges, cudaStream_t st,
                        const uint32_t *d_L) {
    if (L == 0) return;
    k_tile_ranges<<<grid_for(L, 256), 256, 0, st>>>(tkey_sorted, L, d_L, ranges);
}

__global__ void k_clamp_pairs(uint32_t *small, int total, int clamped, int overflow, const ChainSizes *dsz) {
    const uint32_t L = small[total], cap = dsz->L_cap;
    small[clamped] = L < cap ? L : cap;
    small[overflow] = L > cap ? 1u : 0u;
}

void launch_clamp_pairs(uint32_t *small, int total, int clamped, int overflow, const ChainSizes *dsz,
                        cudaStream_t st) {
    k_clamp_pairs<<<1, 1, 0, st>>>(small, total, clamped, overflow, dsz);
}

}  // namespace dgs
