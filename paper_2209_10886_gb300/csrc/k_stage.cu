// One stage of the sweep schedule: all subdomain solves that the schedule
// makes independent run in this single launch (paper Sections 4-5), with the
// assembly of the local right-hand sides from the volume source and the
// incoming interface data (Eq. subPbm, subPbmLifting) in the prologue and the
// transmission of the outgoing traces to the neighbours in the epilogue.
//
// Local solve with the stored factors X_r (k_factor.cu):
//     forward   y_1 = X_1 b_1,        y_r = X_r (b_r + y_{r-1})
//     backward  u_my = y_my,          u_r = y_r + X_r u_{r+1}
// X_r is complex symmetric, so y = X v is computed column-wise from the
// row-major storage (thread = output column, coalesced rows).  X is streamed
// from HBM through a multi-stage shared-memory ring filled with cp.async;
// the first X of the backward pass follows the last forward one in the same
// stream of chunks, so the copy engine never idles between the two passes.
//
// Outgoing data toward the neighbour across side s (scaled form of
// (-d_{n_{i,j}} - T) u_i):  G_out = ca * G_in + cb * u_p  with the edge's
// coefficients, written as  dst = base - sub + G_out  (see StageArgs).
#include "helm_internal.cuh"

namespace {

constexpr int ST = 512;       // threads per CTA
constexpr int NSTAGE = 4;     // pipeline depth

__device__ __forceinline__ void cp_async16(void* smem, const void* gmem) {
    unsigned s = (unsigned)__cvta_generic_to_shared(smem);
    asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(s), "l"(gmem) : "memory");
}
__device__ __forceinline__ void cp_async_commit() { asm volatile("cp.async.commit_group;\n" ::: "memory"); }
template <int N> __device__ __forceinline__ void cp_async_wait() {
    asm volatile("cp.async.wait_group %0;\n" ::"n"(N) : "memory");
}

// BASIS = true: the NR right-hand sides of a CTA are unit data at consecutive
// interface boundary points (columns of the boundary operator K, see StageArgs).
template <typename R, int NR, bool BASIS>
__global__ void __launch_bounds__(ST) stage_kernel(StageArgs<R> a, int rows_per_chunk) {
    using T = Cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int s = BASIS ? blockIdx.x : a.subs[blockIdx.x];
    const SubDev sd = a.subtab[s];
    const int mx = sd.mx, my = sd.my, ldx = sd.ldx;
    const int rhs0 = blockIdx.y * NR;                    // first RHS (workspace slot) of this CTA
    const int e0 = BASIS ? a.col0 + rhs0 : 0;            // first boundary point (basis mode)
    if (BASIS && e0 >= sd.Lb) return;
    const int nr = BASIS ? min(NR, sd.Lb - e0) : min(NR, a.nrhs - rhs0);
    const int tid = threadIdx.x;
    const int NC = (mx + 31) & ~31;
    const int G = ST / NC;
    const int col = tid % NC, grp = tid / NC;
    const bool worker = grp < G && col < mx;
    const bool lead = grp == 0 && col < mx;       // owns column `col` of the solution
    const int Rch = rows_per_chunk;
    const int nq = (mx + Rch - 1) / Rch;
    const int Q = (2 * my - 1) * nq;
    // boundary arrays per RHS: W[my] | E[my] | S[mx] | N[mx]
    const int L = 2 * (mx + my);
    const int boff[4] = {0, my, 2 * my, 2 * my + mx};

    // shared memory: NSTAGE chunks | v[NR][NC] | part[NR*ST] | binc[NR][L] | ub[NR][L]
    T* stg = reinterpret_cast<T*>(smem_raw);
    const size_t chunk_elems = (size_t)Rch * ldx;
    T* v = stg + (size_t)NSTAGE * chunk_elems;
    T* part = v + (size_t)NR * NC;
    T* binc = part + (size_t)NR * ST;
    T* ub = binc + (size_t)NR * L;

    const long long N = (long long)a.nx * a.ny;
    const T* Xs = a.X + sd.xoff;

    auto issue = [&](int t) {
        if (t < Q) {
            int r, q;
            if (t < my * nq) { r = t / nq; q = t - r * nq; }
            else { int tb = t - my * nq; r = my - 2 - tb / nq; q = tb % nq; }
            const int rows = min(Rch, mx - q * Rch);
            const T* src = Xs + (long long)r * mx * ldx + (long long)q * Rch * ldx;
            T* dst = stg + (size_t)(t % NSTAGE) * chunk_elems;
            const int pieces = (int)((size_t)rows * ldx * sizeof(T) / 16);
            const char* sg = reinterpret_cast<const char*>(src);
            char* dg = reinterpret_cast<char*>(dst);
            for (int pc = tid; pc < pieces; pc += ST) cp_async16(dg + 16 * (size_t)pc, sg + 16 * (size_t)pc);
        }
        cp_async_commit();
    };
    auto gin = [&](int k, long long idx) -> T {
        T g = a.gin0 ? a.gin0[(long long)(rhs0 + k) * a.ntrace + idx] : czero<T>();
        if (a.gin1) g = cadd(g, a.gin1[(long long)(rhs0 + k) * a.ntrace + idx]);
        return g;
    };
    // incoming-data part of the local right-hand side at node (r, c) (from shared memory)
    auto bterm = [&](int r, int c, int k) -> T {
        const T* bk = binc + (size_t)k * L;
        T b = czero<T>();
        if (c == 0) b = cadd(b, bk[boff[SW] + r]);
        if (c == mx - 1) b = cadd(b, bk[boff[SE] + r]);
        if (r == 0) b = cadd(b, bk[boff[SS] + c]);
        if (r == my - 1) b = cadd(b, bk[boff[SN] + c]);
        return b;
    };
    auto src_row = [&](int r, int c, int k) -> double2 {
        return a.r[(long long)(rhs0 + k) * N + (long long)(sd.y0 + r) * a.nx + sd.x0 + c];
    };
    double rsc[NR], zsc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        rsc[k] = (a.rscale && k < nr) ? a.rscale[rhs0 + k] : 1.0;
        zsc[k] = (a.zscale && k < nr) ? a.zscale[rhs0 + k] : 1.0;
    }
    auto scaled = [&](double2 rv, int k) -> T {
        const double sc = rsc[k];
        return from_c128<T>(make_double2(rv.x * sc, rv.y * sc));
    };
    // row r of the solution is final: keep the boundary values, write the volume output
    auto finish_row = [&](int r, int c, int k, T u) {
        T* uk = ub + (size_t)k * L;
        if (c == 0) uk[boff[SW] + r] = u;
        if (c == mx - 1) uk[boff[SE] + r] = u;
        if (r == 0) uk[boff[SS] + c] = u;
        if (r == my - 1) uk[boff[SN] + c] = u;
        if (!BASIS && a.z) {
            const double sc = zsc[k];
            const double2 zu = to_c128(u);
            a.z[(long long)(rhs0 + k) * N + (long long)(sd.y0 + r) * a.nx + sd.x0 + c] =
                make_double2(zu.x * sc, zu.y * sc);
        }
    };

    // ---- prologue: start the copies; incoming terms G_in/(1-beta) into shared memory
    for (int t = 0; t < NSTAGE - 1; ++t) issue(t);
    for (int idx = tid; idx < NR * L; idx += ST) {
        const int k = idx / L, e = idx - k * L;
        const int side = e < my ? SW : e < 2 * my ? SE : e < 2 * my + mx ? SS : SN;
        const int pt = e - boff[side];
        T b = czero<T>();
        if (BASIS) {
            // unit datum at boundary point e0 + k (an interface side's point)
            if (k < nr && sd.bo[side] >= 0 && sd.bo[side] + pt == e0 + k) b = mk((R)1, (R)0);
        } else if (k < nr && sd.tin[side] >= 0 && (a.gin0 || a.gin1)) {
            const long long ti = sd.tin[side] + pt;
            b = cmul(gin(k, ti), a.tc[ti].cin);
        }
        binc[idx] = b;
    }
    __syncthreads();
    for (int idx = tid; idx < NR * mx; idx += ST) {
        const int k = idx / mx, c = idx - k * mx;
        T b = czero<T>();
        if (k < nr) {
            b = bterm(0, c, k);
            if (!BASIS && a.src) b = cadd(b, scaled(src_row(0, c, k), k));
        }
        v[k * NC + c] = b;
    }
    // one-row-ahead register prefetch (raw loads; consumed at the end of the next row)
    double2 rnext[NR];
    T ynext[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) { rnext[k] = make_double2(0.0, 0.0); ynext[k] = czero<T>(); }
    if (!BASIS && lead && a.src && my > 1) {
#pragma unroll
        for (int k = 0; k < NR; ++k)
            if (k < nr) rnext[k] = src_row(1, col, k);
    }

    T acc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) acc[k] = czero<T>();
    T* yw = a.yws + sd.yoff;

    for (int t = 0; t < Q; ++t) {
        cp_async_wait<NSTAGE - 2>();
        __syncthreads();
        issue(t + NSTAGE - 1);
        int r, q;
        bool fwd;
        if (t < my * nq) { r = t / nq; q = t - r * nq; fwd = true; }
        else { int tb = t - my * nq; r = my - 2 - tb / nq; q = tb % nq; fwd = false; }
        const int rows = min(Rch, mx - q * Rch);
        const T* S = stg + (size_t)(t % NSTAGE) * chunk_elems;
        if (worker) {
            const T* vq = v + q * Rch;
#pragma unroll 4
            for (int jj = grp; jj < rows; jj += G) {
                const T xv = S[(size_t)jj * ldx + col];
#pragma unroll
                for (int k = 0; k < NR; ++k) acc[k] = cfma(xv, vq[k * NC + jj], acc[k]);
            }
        }
        if (q == nq - 1) {
            if (worker) {
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    part[(size_t)(grp * NR + k) * NC + col] = acc[k];
                    acc[k] = czero<T>();
                }
            }
            __syncthreads();
            if (lead) {
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    if (k >= nr) break;
                    T sum = part[(size_t)k * NC + col];
                    for (int g2 = 1; g2 < G; ++g2) sum = cadd(sum, part[(size_t)(g2 * NR + k) * NC + col]);
                    T* ywk = yw + (long long)(rhs0 + k) * a.wstride;
                    T nv;
                    if (fwd) {
                        if (r < my - 1) {
                            ywk[(long long)r * mx + col] = sum;                   // y_r
                            T b = bterm(r + 1, col, k);
                            if (!BASIS && a.src) b = cadd(b, scaled(rnext[k], k));
                            nv = cadd(b, sum);                                     // b_{r+1} + y_r
                            if (!BASIS && a.src && r + 2 < my) rnext[k] = src_row(r + 2, col, k);
                            if (r + 2 == my) ynext[k] = sum;                       // y_{my-1} for the first backward row
                        } else {
                            finish_row(r, col, k, sum);                            // u_my = y_my
                            nv = sum;
                        }
                    } else {
                        const T u = cadd(ynext[k], sum);                          // u_r = y_r + X_r u_{r+1}
                        finish_row(r, col, k, u);
                        nv = u;
                        if (r >= 1) ynext[k] = ywk[(long long)(r - 1) * mx + col];
                    }
                    v[k * NC + col] = nv;
                }
            }
            // the next iteration's barrier orders these writes of v before any read
        }
    }
    cp_async_wait<0>();
    __syncthreads();

    if (BASIS) {
        // row e0 + k of K = boundary values of the response to the unit datum
        // (K is symmetric: K = the interface-boundary block of the local inverse)
        for (int idx = tid; idx < NR * L; idx += ST) {
            const int k = idx / L, e = idx - k * L;
            if (k >= nr) continue;
            const int side = e < my ? SW : e < 2 * my ? SE : e < 2 * my + mx ? SS : SN;
            if (sd.bo[side] < 0) continue;
            const int pt = e - boff[side];
            a.K[sd.koff + (long long)(e0 + k) * sd.Lb + sd.bo[side] + pt] = ub[idx];
        }
        return;
    }
    // ---- epilogue: outgoing data G_out = ca G_in + cb u_p toward the masked sides
    if (a.mask) {
        for (int idx = tid; idx < NR * L; idx += ST) {
            const int k = idx / L, e = idx - k * L;
            if (k >= nr) continue;
            const int side = e < my ? SW : e < 2 * my ? SE : e < 2 * my + mx ? SS : SN;
            if (!(a.mask & (1 << side)) || sd.tin[side] < 0) continue;
            const int pt = e - boff[side];
            const long long in = sd.tin[side] + pt, out = sd.tout[side] + pt;
            const TraceCoef<T> c = a.tc[in];
            T g = cfma(c.cb, ub[idx], cmul(c.ca, gin(k, in)));
            const long long o = (long long)(rhs0 + k) * a.ntrace + out;
            if (a.base) g = cadd(g, a.base[o]);
            if (a.sub) g = csub(g, a.sub[o]);
            a.dst[o] = g;
            if (a.dst2) a.dst2[o] = g;
        }
    }
}

template <typename R, int NR, bool BASIS>
cudaError_t launch_nr(const StageArgs<R>& a, int nactive, int ny_blocks, int max_mx, int max_my, cudaStream_t st) {
    using T = Cx<R>;
    const int maxldx = sizeof(T) == 8 ? ((max_mx + 1) & ~1) : max_mx;
    const int NC = (max_mx + 31) & ~31;
    const int G = ST / NC;
    // v[NR][NC] plus part[G][NR][NC]; a narrower subdomain in the same launch
    // has more row groups, but G*NC <= ST always
    const size_t fixed = (size_t)NR * NC * sizeof(T) + (size_t)NR * ST * sizeof(T) +
                         2 * (size_t)NR * 2 * (max_mx + max_my) * sizeof(T);
    const size_t budget = 227 * 1024 - 2048;
    if (fixed >= budget) return cudaErrorInvalidValue;
    size_t per_chunk_max = (budget - fixed) / NSTAGE;
    int rows = (int)(per_chunk_max / ((size_t)maxldx * sizeof(T)));
    rows = min(rows, max_mx);
    if (rows >= G) rows -= rows % G;
    if (rows < 1) return cudaErrorInvalidValue;
    const size_t smem = fixed + (size_t)NSTAGE * rows * maxldx * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<R, NR, BASIS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(nactive, ny_blocks);
    count_launch();
    stage_kernel<R, NR, BASIS><<<grid, ST, smem, st>>>(a, rows);
    return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_stage(const StageArgs<R>& a, int nactive, int max_mx, int max_my, cudaStream_t st) {
    if (nactive == 0) return cudaSuccess;
    if (max_mx > ST) return cudaErrorInvalidValue;
    if (a.nrhs >= 4) return launch_nr<R, 4, false>(a, nactive, (a.nrhs + 3) / 4, max_mx, max_my, st);
    if (a.nrhs >= 2) return launch_nr<R, 2, false>(a, nactive, (a.nrhs + 1) / 2, max_mx, max_my, st);
    return launch_nr<R, 1, false>(a, nactive, a.nrhs, max_mx, max_my, st);
}

template <typename R>
cudaError_t launch_basis(const StageArgs<R>& a, int nsub, int ncols, int max_mx, int max_my, cudaStream_t st) {
    if (max_mx > ST) return cudaErrorInvalidValue;
    return launch_nr<R, 4, true>(a, nsub, (ncols + 3) / 4, max_mx, max_my, st);
}
template cudaError_t launch_basis<float>(const StageArgs<float>&, int, int, int, int, cudaStream_t);
template cudaError_t launch_basis<double>(const StageArgs<double>&, int, int, int, int, cudaStream_t);

template cudaError_t launch_stage<float>(const StageArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_stage<double>(const StageArgs<double>&, int, int, int, cudaStream_t);
