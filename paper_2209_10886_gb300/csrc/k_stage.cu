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

template <typename R, int NR>
__global__ void __launch_bounds__(ST) stage_kernel(StageArgs<R> a, int rows_per_chunk) {
    using T = Cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    const int s = a.subs[blockIdx.x];
    const SubDev sd = a.subtab[s];
    const int mx = sd.mx, my = sd.my, ldx = sd.ldx;
    const int rhs0 = blockIdx.y * NR;
    const int nr = min(NR, a.nrhs - rhs0);
    const int tid = threadIdx.x;
    const int NC = (mx + 31) & ~31;
    const int G = ST / NC;
    const int col = tid % NC, grp = tid / NC;
    const bool worker = grp < G && col < mx;
    const int Rch = rows_per_chunk;
    const int nq = (mx + Rch - 1) / Rch;
    const int Q = (2 * my - 1) * nq;

    // shared memory: NSTAGE chunks | v[NR][NC] | part[G][NR][NC]
    T* stg = reinterpret_cast<T*>(smem_raw);
    const size_t chunk_elems = (size_t)Rch * ldx;
    T* v = stg + (size_t)NSTAGE * chunk_elems;
    T* part = v + (size_t)NR * NC;

    const long long N = (long long)a.nx * a.ny;
    const T* Xs = a.X + sd.xoff;

    auto chunk_src = [&](int t, int& rows) -> const T* {
        int r, q;
        if (t < my * nq) { r = t / nq; q = t - r * nq; }
        else { int tb = t - my * nq; r = my - 2 - tb / nq; q = tb % nq; }
        rows = min(Rch, mx - q * Rch);
        return Xs + (long long)r * mx * ldx + (long long)q * Rch * ldx;
    };
    auto issue = [&](int t) {
        if (t < Q) {
            int rows;
            const T* src = chunk_src(t, rows);
            T* dst = stg + (size_t)(t % NSTAGE) * chunk_elems;
            const int pieces = (int)((size_t)rows * ldx * sizeof(T) / 16);
            const char* sg = reinterpret_cast<const char*>(src);
            char* dg = reinterpret_cast<char*>(dst);
            for (int pc = tid; pc < pieces; pc += ST) cp_async16(dg + 16 * (size_t)pc, sg + 16 * (size_t)pc);
        }
        cp_async_commit();
    };

    // incoming data at trace index idx for RHS k (in0 + in1)
    auto gin = [&](int k, long long idx) -> T {
        T g = a.gin0 ? a.gin0[(long long)(rhs0 + k) * a.ntrace + idx] : czero<T>();
        if (a.gin1) g = cadd(g, a.gin1[(long long)(rhs0 + k) * a.ntrace + idx]);
        return g;
    };
    // local right-hand side of row r, column c, RHS k
    auto rhs = [&](int r, int c, int k) -> T {
        T b = czero<T>();
        if (a.src) {
            const double sc = a.rscale ? a.rscale[rhs0 + k] : 1.0;
            const double2 rv = a.r[(long long)(rhs0 + k) * N + (long long)(sd.y0 + r) * a.nx + sd.x0 + c];
            b = from_c128<T>(make_double2(rv.x * sc, rv.y * sc));
        }
        if (c == 0 && sd.tin[SW] >= 0) b = cfma(gin(k, sd.tin[SW] + r), a.tc[sd.tin[SW] + r].cin, b);
        if (c == mx - 1 && sd.tin[SE] >= 0) b = cfma(gin(k, sd.tin[SE] + r), a.tc[sd.tin[SE] + r].cin, b);
        if (r == 0 && sd.tin[SS] >= 0) b = cfma(gin(k, sd.tin[SS] + c), a.tc[sd.tin[SS] + c].cin, b);
        if (r == my - 1 && sd.tin[SN] >= 0) b = cfma(gin(k, sd.tin[SN] + c), a.tc[sd.tin[SN] + c].cin, b);
        return b;
    };
    auto emit = [&](int side, int kpt, T u, int k) {
        const long long in = sd.tin[side] + kpt, out = sd.tout[side] + kpt;
        const TraceCoef<T> c = a.tc[in];
        T g = cfma(c.cb, u, cmul(c.ca, gin(k, in)));
        const long long o = (long long)(rhs0 + k) * a.ntrace + out;
        if (a.base) g = cadd(g, a.base[o]);
        if (a.sub) g = csub(g, a.sub[o]);
        a.dst[o] = g;
        if (a.dst2) a.dst2[o] = g;
    };
    // row r of the solution is final (backward pass, or the last forward row)
    auto finish_row = [&](int r, int c, int k, T u) {
        if (a.mask) {
            if ((a.mask & (1 << SW)) && c == 0 && sd.tin[SW] >= 0) emit(SW, r, u, k);
            if ((a.mask & (1 << SE)) && c == mx - 1 && sd.tin[SE] >= 0) emit(SE, r, u, k);
            if ((a.mask & (1 << SS)) && r == 0 && sd.tin[SS] >= 0) emit(SS, c, u, k);
            if ((a.mask & (1 << SN)) && r == my - 1 && sd.tin[SN] >= 0) emit(SN, c, u, k);
        }
        if (a.z) {
            const double sc = a.zscale ? a.zscale[rhs0 + k] : 1.0;
            double2 zu = to_c128(u);
            a.z[(long long)(rhs0 + k) * N + (long long)(sd.y0 + r) * a.nx + sd.x0 + c] =
                make_double2(zu.x * sc, zu.y * sc);
        }
    };

    // prologue: start the copies, build v = b_1
    for (int t = 0; t < NSTAGE - 1; ++t) issue(t);
    for (int idx = tid; idx < NR * mx; idx += ST) {
        const int k = idx / mx, c = idx - k * mx;
        v[k * NC + c] = k < nr ? rhs(0, c, k) : czero<T>();
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
                    part[((size_t)grp * NR + k) * NC + col] = acc[k];
                    acc[k] = czero<T>();
                }
            }
            __syncthreads();
            if (grp == 0 && col < mx) {
                for (int k = 0; k < nr; ++k) {
                    T sum = part[(size_t)k * NC + col];
                    for (int g2 = 1; g2 < G; ++g2) sum = cadd(sum, part[((size_t)g2 * NR + k) * NC + col]);
                    T* ywk = yw + (long long)(rhs0 + k) * a.wstride;
                    T nv;
                    if (fwd) {
                        ywk[(long long)r * mx + col] = sum;                       // y_r
                        if (r < my - 1) {
                            nv = cadd(rhs(r + 1, col, k), sum);                  // b_{r+1} + y_r
                        } else {
                            finish_row(r, col, k, sum);                           // u_my = y_my
                            nv = sum;
                        }
                    } else {
                        const T u = cadd(ywk[(long long)r * mx + col], sum);     // u_r = y_r + X_r u_{r+1}
                        finish_row(r, col, k, u);
                        nv = u;
                    }
                    v[k * NC + col] = nv;
                }
            }
            // the next iteration's barrier orders these writes of v before any read
        }
    }
    cp_async_wait<0>();
}

template <typename R, int NR>
cudaError_t launch_nr(const StageArgs<R>& a, int nactive, int max_mx, cudaStream_t st) {
    using T = Cx<R>;
    const int maxldx = sizeof(T) == 8 ? ((max_mx + 1) & ~1) : max_mx;
    const int NC = (max_mx + 31) & ~31;
    const int G = ST / NC;
    // v[NR][NC] plus part[G][NR][NC]; a narrower subdomain in the same launch
    // has more row groups, but G*NC <= ST always
    const size_t fixed = (size_t)NR * NC * sizeof(T) + (size_t)NR * ST * sizeof(T);
    const size_t budget = 227 * 1024 - 2048;
    if (fixed >= budget) return cudaErrorInvalidValue;
    size_t per_chunk_max = (budget - fixed) / NSTAGE;
    int rows = (int)(per_chunk_max / ((size_t)maxldx * sizeof(T)));
    rows = min(rows, max_mx);
    if (rows >= G) rows -= rows % G;
    if (rows < 1) return cudaErrorInvalidValue;
    const size_t smem = fixed + (size_t)NSTAGE * rows * maxldx * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(nactive, (a.nrhs + NR - 1) / NR);
    stage_kernel<R, NR><<<grid, ST, smem, st>>>(a, rows);
    return cudaGetLastError();
}

}  // namespace

template <typename R>
cudaError_t launch_stage(const StageArgs<R>& a, int nactive, int max_mx, cudaStream_t st) {
    if (nactive == 0) return cudaSuccess;
    if (max_mx > ST) return cudaErrorInvalidValue;
    if (a.nrhs >= 4) return launch_nr<R, 4>(a, nactive, max_mx, st);
    if (a.nrhs >= 2) return launch_nr<R, 2>(a, nactive, max_mx, st);
    return launch_nr<R, 1>(a, nactive, max_mx, st);
}

template cudaError_t launch_stage<float>(const StageArgs<float>&, int, int, cudaStream_t);
template cudaError_t launch_stage<double>(const StageArgs<double>&, int, int, cudaStream_t);
