// One stage of the sweep schedule that needs full subdomain solves (the
// liftings of Eq. subPbmLifting and the reconstruction with the final
// interface data): all subdomains of the stage run in this single launch
// (paper Sections 4-5), with the assembly of the local right-hand sides from
// the volume source and the incoming data (Eq. subPbm) in the prologue and the
// transmission of the outgoing traces to the neighbours in the epilogue.
//
// Local solve with the stored factors X_r (k_factor.cu):
//     forward   y_1 = X_1 b_1,        y_r = X_r (b_r + y_{r-1})
//     backward  u_my = y_my,          u_r = y_r + X_r u_{r+1}
// X_r is complex symmetric, so y = X v is computed column-wise from the
// row-major storage: one consumer thread per output column, coalesced rows in
// shared memory, four independent partial sums.  X is streamed from HBM by
// bulk (TMA) copies that one producer thread issues into a ring of shared
// memory slots guarded by full/empty mbarriers; the first X of the backward
// pass follows the last forward one in the same stream of chunks.  Every
// mbarrier wait is bounded in time; on expiry the kernel records HELM_ERR_TIMEOUT
// in a device flag, drains its own copies and returns.
//
// Outgoing data toward the neighbour across side s (scaled form of
// (-d_{n_{i,j}} - T) u_i):  G_out = ca * G_in + cb * u_p  with the edge's
// coefficients, written as  dst = base - sub + G_out  (see StageArgs).
#include "helm_internal.cuh"

namespace {

constexpr int MAXNS = 8;                        // ring slots (upper bound)
constexpr long long WAIT_LIMIT = 2000000000LL;  // cycles (~1 s) before a wait gives up

__device__ __forceinline__ unsigned smem_addr(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }

__device__ __forceinline__ void mbar_init(unsigned long long* b, unsigned count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;\n" ::"r"(smem_addr(b)), "r"(count) : "memory");
}
__device__ __forceinline__ void mbar_arrive(unsigned long long* b) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];\n" ::"r"(smem_addr(b)) : "memory");
}
__device__ __forceinline__ void mbar_expect_tx(unsigned long long* b, unsigned bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_addr(b)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for the phase with this parity, at most WAIT_LIMIT cycles
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity) {
    if (mbar_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!mbar_try(b, parity))
        if (clock64() - t0 > WAIT_LIMIT) return false;
    return true;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void consumer_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;\n" ::"r"(nthreads) : "memory");
}

// BASIS = true: the NR right-hand sides of a CTA are unit data at consecutive
// interface boundary points (columns of the boundary operator K, see StageArgs).
template <typename R, int NR, bool BASIS>
__global__ void __launch_bounds__(NR <= 4 ? 544 : 288) stage_kernel(StageArgs<R> a, int rows_per_chunk, int nslots,
                                                                  int cwarps, int ngroups) {
    using T = Cx<R>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long full_bar[MAXNS], empty_bar[MAXNS];
    __shared__ int abort_flag;

    const int s = BASIS ? blockIdx.x : a.subs[blockIdx.x];
    const SubDev sd = a.subtab[s];
    const int mx = sd.mx, my = sd.my, ldx = sd.ldx;
    const int rhs0 = blockIdx.y * NR;                    // first RHS (workspace slot) of this CTA
    const int e0 = BASIS ? a.col0 + rhs0 : 0;            // first boundary point (basis mode)
    if (BASIS && e0 >= sd.Lb) return;
    const int nr = BASIS ? min(NR, sd.Lb - e0) : min(NR, a.nrhs - rhs0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // consumers: ngroups groups of cwarps warps; thread (grp, col) sums the rows
    // grp, grp + ngroups, ... of every chunk for output column col
    const int ncons = 32 * cwarps * ngroups;
    const bool producer = warp == cwarps * ngroups;
    const int col = tid % (32 * cwarps);
    const int grp = tid / (32 * cwarps);
    const bool worker = !producer && col < mx;
    const bool owner = worker && grp == 0;               // finishes column col of every row
    const int Rch = rows_per_chunk;
    const int nq = (mx + Rch - 1) / Rch;
    const int Q = (2 * my - 1) * nq;
    const int mxp = 32 * cwarps;
    // boundary arrays per RHS: W[my] | E[my] | S[mx] | N[mx]
    const int L = 2 * (mx + my);
    auto boff = [&](int side) { return side < 2 ? side * my : 2 * my + (side - 2) * mx; };

    // dynamic shared memory: ring[nslots][Rch*ldx] | v[2][NR][mxp] | binc[NR][L] | ub[NR][L]
    T* ring = reinterpret_cast<T*>(smem_raw);
    const size_t slot_elems = (size_t)Rch * ldx;
    T* vbuf = ring + (size_t)nslots * slot_elems;
    T* binc = vbuf + 2 * (size_t)NR * mxp;
    T* ub = binc + (size_t)NR * L;
    T* part = ub + (size_t)NR * L;                       // [ngroups-1][NR][mxp] row-group partial sums

    const long long N = (long long)a.nx * a.ny;
    const T* Xs = a.X + sd.xoff;

    auto gin = [&](int k, long long idx) -> T {
        T g = a.gin0 ? a.gin0[(long long)(rhs0 + k) * a.ntrace + idx] : czero<T>();
        if (a.gin1) g = cadd(g, a.gin1[(long long)(rhs0 + k) * a.ntrace + idx]);
        return g;
    };
    auto bterm = [&](int r, int c, int k) -> T {
        const T* bk = binc + (size_t)k * L;
        T b = czero<T>();
        if (c == 0) b = cadd(b, bk[boff(SW) + r]);
        if (c == mx - 1) b = cadd(b, bk[boff(SE) + r]);
        if (r == 0) b = cadd(b, bk[boff(SS) + c]);
        if (r == my - 1) b = cadd(b, bk[boff(SN) + c]);
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
    auto scaled = [&](double2 rv, int k) -> T { return from_c128<T>(make_double2(rv.x * rsc[k], rv.y * rsc[k])); };
    auto finish_row = [&](int r, int c, int k, T u) {
        T* uk = ub + (size_t)k * L;
        if (c == 0) uk[boff(SW) + r] = u;
        if (c == mx - 1) uk[boff(SE) + r] = u;
        if (r == 0) uk[boff(SS) + c] = u;
        if (r == my - 1) uk[boff(SN) + c] = u;
        if (!BASIS && a.z) {
            const double2 zu = to_c128(u);
            a.z[(long long)(rhs0 + k) * N + (long long)(sd.y0 + r) * a.nx + sd.x0 + c] =
                make_double2(zu.x * zsc[k], zu.y * zsc[k]);
        }
    };

    // ---- prologue: barriers, incoming terms G_in/(1-beta) into shared memory, v = b_1
    if (tid == 0) {
        for (int i = 0; i < nslots; ++i) {
            mbar_init(&full_bar[i], 1);
            mbar_init(&empty_bar[i], cwarps * ngroups);
        }
        abort_flag = 0;
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    for (int idx = tid; idx < NR * L; idx += blockDim.x) {
        const int k = idx / L, e = idx - k * L;
        const int side = e < my ? SW : e < 2 * my ? SE : e < 2 * my + mx ? SS : SN;
        const int pt = e - boff(side);
        T b = czero<T>();
        if (BASIS) {
            if (k < nr && sd.bo[side] >= 0 && sd.bo[side] + pt == e0 + k) b = mk((R)1, (R)0);
        } else if (k < nr && sd.tin[side] >= 0 && (a.gin0 || a.gin1)) {
            const long long ti = sd.tin[side] + pt;
            b = cmul(gin(k, ti), a.tc[ti].cin);
        }
        binc[idx] = b;
    }
    __syncthreads();
    for (int idx = tid; idx < NR * mxp; idx += blockDim.x) {
        const int k = idx / mxp, c = idx - k * mxp;
        T b = czero<T>();
        if (k < nr && c < mx) {
            b = bterm(0, c, k);
            if (!BASIS && a.src) b = cadd(b, scaled(src_row(0, c, k), k));
        }
        vbuf[idx] = b;
    }
    __syncthreads();

    if (producer) {
        // ---- producer: one thread streams every chunk of X_1..X_my, X_{my-1}..X_1
        if (lane == 0) {
            int r = 0, q = 0, slot = 0;
            unsigned ph = 0;
            bool fwd = true;
            int issued = 0;
            for (int t = 0; t < Q; ++t) {
                if (t >= nslots && !mbar_wait(&empty_bar[slot], ph ^ 1u)) {
                    abort_flag = 1;
                    if (a.err) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
                    break;
                }
                if (*((volatile int*)&abort_flag)) break;
                const int rows = min(Rch, mx - q * Rch);
                const unsigned bytes = (unsigned)((size_t)rows * ldx * sizeof(T));
                mbar_expect_tx(&full_bar[slot], bytes);
                bulk_copy(ring + (size_t)slot * slot_elems, Xs + (long long)r * mx * ldx + (long long)q * Rch * ldx,
                          bytes, &full_bar[slot]);
                ++issued;
                if (++slot == nslots) { slot = 0; ph ^= 1u; }
                if (++q == nq) {
                    q = 0;
                    if (fwd) { if (++r == my) { fwd = false; r = my - 2; } }
                    else --r;
                }
            }
            if (*((volatile int*)&abort_flag)) {
                // drain: wait (bounded) for every copy this CTA issued before leaving
                for (int t = max(0, issued - nslots); t < issued; ++t)
                    mbar_wait(&full_bar[t % nslots], (unsigned)((t / nslots) & 1));
            }
        }
    } else {
        // ---- consumers: y = X v column-wise, one thread per column
        double2 rnext[NR];
        T ynext[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) { rnext[k] = make_double2(0.0, 0.0); ynext[k] = czero<T>(); }
        if (!BASIS && owner && a.src && my > 1) {
#pragma unroll
            for (int k = 0; k < NR; ++k)
                if (k < nr) rnext[k] = src_row(1, col, k);
        }
        T* yw = a.yws + sd.yoff;
        int slot = 0;
        unsigned ph = 0;
        int cur = 0;                                      // v buffer holding the current step's input
        const int nsteps = 2 * my - 1;
        for (int step = 0; step < nsteps; ++step) {
            const bool fwd = step < my;
            const int r = fwd ? step : 2 * my - 2 - step;
            const T* v = vbuf + (size_t)cur * NR * mxp;
            // independent partial sums: 4 per RHS for few RHS, else the RHS themselves
            constexpr int U = NR >= 8 ? 1 : 4;
            T acc[NR][U];
#pragma unroll
            for (int k = 0; k < NR; ++k)
#pragma unroll
                for (int u = 0; u < U; ++u) acc[k][u] = czero<T>();
            for (int q = 0; q < nq; ++q) {
                if (!mbar_wait(&full_bar[slot], ph)) {
                    abort_flag = 1;
                    if (a.err) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
                }
                if (worker && !*((volatile int*)&abort_flag)) {
                    const T* S = ring + (size_t)slot * slot_elems + col;
                    const T* vq = v + q * Rch;
                    const int rows = min(Rch, mx - q * Rch);
                    const int G = ngroups;
                    int jj = grp;
                    for (; jj + 3 * G < rows; jj += 4 * G) {
                        const T x0 = S[(size_t)(jj + 0 * G) * ldx], x1 = S[(size_t)(jj + 1 * G) * ldx];
                        const T x2 = S[(size_t)(jj + 2 * G) * ldx], x3 = S[(size_t)(jj + 3 * G) * ldx];
#pragma unroll
                        for (int k = 0; k < NR; ++k) {
                            const T* vk = vq + k * mxp + jj;
                            acc[k][0 % U] = cfma(x0, vk[0 * G], acc[k][0 % U]);
                            acc[k][1 % U] = cfma(x1, vk[1 * G], acc[k][1 % U]);
                            acc[k][2 % U] = cfma(x2, vk[2 * G], acc[k][2 % U]);
                            acc[k][3 % U] = cfma(x3, vk[3 * G], acc[k][3 % U]);
                        }
                    }
                    for (; jj < rows; jj += G) {
                        const T x0 = S[(size_t)jj * ldx];
#pragma unroll
                        for (int k = 0; k < NR; ++k) acc[k][0] = cfma(x0, vq[k * mxp + jj], acc[k][0]);
                    }
                }
                __syncwarp();
                if (lane == 0) mbar_arrive(&empty_bar[slot]);
                if (++slot == nslots) { slot = 0; ph ^= 1u; }
            }
            if (ngroups > 1) {
                // row groups 1.. hand their partial sums to group 0
                if (worker && grp > 0) {
#pragma unroll
                    for (int k = 0; k < NR; ++k) {
                        T sum = acc[k][0];
#pragma unroll
                        for (int u = 1; u < U; ++u) sum = cadd(sum, acc[k][u]);
                        part[((size_t)(grp - 1) * NR + k) * mxp + col] = sum;
                    }
                }
                consumer_sync(ncons);
                if (owner) {
#pragma unroll
                    for (int k = 0; k < NR; ++k)
                        for (int g2 = 1; g2 < ngroups; ++g2)
                            acc[k][0] = cadd(acc[k][0], part[((size_t)(g2 - 1) * NR + k) * mxp + col]);
                }
            }
            T* vn = vbuf + (size_t)(cur ^ 1) * NR * mxp;
            if (owner) {
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    if (k >= nr) break;
                    T sum = acc[k][0];
#pragma unroll
                    for (int u = 1; u < U; ++u) sum = cadd(sum, acc[k][u]);
                    T* ywk = yw + (long long)(rhs0 + k) * a.wstride;
                    T nv;
                    if (fwd) {
                        if (r < my - 1) {
                            ywk[(long long)r * mx + col] = sum;                   // y_r
                            T b = bterm(r + 1, col, k);
                            if (!BASIS && a.src) b = cadd(b, scaled(rnext[k], k));
                            nv = cadd(b, sum);                                     // b_{r+1} + y_r
                            if (!BASIS && a.src && r + 2 < my) rnext[k] = src_row(r + 2, col, k);
                            if (r + 2 == my) ynext[k] = sum;                       // y_{my-1}
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
                    vn[k * mxp + col] = nv;
                }
            }
            consumer_sync(ncons);
            cur ^= 1;
            if (*((volatile int*)&abort_flag)) break;
        }
    }
    __syncthreads();
    if (abort_flag) return;

    if (BASIS) {
        // row e0 + k of K = boundary values of the response to the unit datum
        for (int idx = tid; idx < NR * L; idx += blockDim.x) {
            const int k = idx / L, e = idx - k * L;
            if (k >= nr) continue;
            const int side = e < my ? SW : e < 2 * my ? SE : e < 2 * my + mx ? SS : SN;
            if (sd.bo[side] < 0) continue;
            const int pt = e - boff(side);
            a.K[sd.koff + (long long)(e0 + k) * sd.Lb + sd.bo[side] + pt] = ub[idx];
        }
        return;
    }
    // ---- epilogue: outgoing data G_out = ca G_in + cb u_p toward the masked sides
    if (a.mask) {
        for (int idx = tid; idx < NR * L; idx += blockDim.x) {
            const int k = idx / L, e = idx - k * L;
            if (k >= nr) continue;
            const int side = e < my ? SW : e < 2 * my ? SE : e < 2 * my + mx ? SS : SN;
            if (!(a.mask & (1 << side)) || sd.tin[side] < 0) continue;
            const int pt = e - boff(side);
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
    const int cwarps = (max_mx + 31) / 32;
    const int mxp = 32 * cwarps;
    // row groups raise the number of consumer warps (latency hiding) for few RHS
    const int ngroups = NR <= 4 ? std::max(1, std::min(4, 16 / cwarps)) : 1;
    const int maxldx = sizeof(T) == 8 ? ((max_mx + 1) & ~1) : max_mx;
    const size_t fixed = 2 * (size_t)NR * mxp * sizeof(T) + 2 * (size_t)NR * 2 * (max_mx + max_my) * sizeof(T) +
                         (size_t)(ngroups - 1) * NR * mxp * sizeof(T);
    const size_t budget = 227 * 1024 - 1024;
    if (fixed >= budget) return cudaErrorInvalidValue;
    // chunk of ~32 KB, a multiple of 4 rows
    int rows = (int)(32768 / ((size_t)maxldx * sizeof(T)));
    rows = std::max(4, rows & ~3);
    rows = std::min(rows, max_mx);
    int nslots = (int)((budget - fixed) / ((size_t)rows * maxldx * sizeof(T)));
    nslots = std::min(nslots, MAXNS);
    if (nslots < 2) return cudaErrorInvalidValue;
    const size_t smem = fixed + (size_t)nslots * rows * maxldx * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<R, NR, BASIS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)smem);
    if (e != cudaSuccess) return e;
    dim3 grid(nactive, ny_blocks);
    count_launch();
    stage_kernel<R, NR, BASIS><<<grid, 32 * (cwarps * ngroups + 1), smem, st>>>(a, rows, nslots, cwarps, ngroups);
    return cudaGetLastError();
}

}  // namespace

// Fixed shared memory of a CTA with NR right-hand sides (the ring needs at least two more slots).
template <typename R, int NR>
static bool stage_fits(int max_mx, int max_my) {
    using T = Cx<R>;
    const int mxp = 32 * ((max_mx + 31) / 32);
    const int maxldx = sizeof(T) == 8 ? ((max_mx + 1) & ~1) : max_mx;
    const int ngroups = NR <= 4 ? std::max(1, std::min(4, 16 / ((max_mx + 31) / 32))) : 1;
    const size_t fixed = 2 * (size_t)NR * mxp * sizeof(T) + 2 * (size_t)NR * 2 * (max_mx + max_my) * sizeof(T) +
                         (size_t)(ngroups - 1) * NR * mxp * sizeof(T);
    int rows = (int)(32768 / ((size_t)maxldx * sizeof(T)));
    rows = std::min(std::max(4, rows & ~3), max_mx);
    return fixed + 2 * (size_t)rows * maxldx * sizeof(T) <= 227 * 1024 - 1024;
}

template <typename R>
cudaError_t launch_stage(const StageArgs<R>& a, int nactive, int max_mx, int max_my, cudaStream_t st) {
    if (nactive == 0) return cudaSuccess;
    if (max_mx > 256) return cudaErrorInvalidValue;
    // as many right-hand sides per CTA as the RHS count and shared memory allow
    if (a.nrhs >= 16 && stage_fits<R, 16>(max_mx, max_my))
        return launch_nr<R, 16, false>(a, nactive, (a.nrhs + 15) / 16, max_mx, max_my, st);
    if (a.nrhs >= 8 && stage_fits<R, 8>(max_mx, max_my))
        return launch_nr<R, 8, false>(a, nactive, (a.nrhs + 7) / 8, max_mx, max_my, st);
    if (a.nrhs >= 4 && stage_fits<R, 4>(max_mx, max_my))
        return launch_nr<R, 4, false>(a, nactive, (a.nrhs + 3) / 4, max_mx, max_my, st);
    if (a.nrhs >= 2 && stage_fits<R, 2>(max_mx, max_my))
        return launch_nr<R, 2, false>(a, nactive, (a.nrhs + 1) / 2, max_mx, max_my, st);
    return launch_nr<R, 1, false>(a, nactive, a.nrhs, max_mx, max_my, st);
}

template <typename R>
cudaError_t launch_basis(const StageArgs<R>& a, int nsub, int ncols, int max_mx, int max_my, cudaStream_t st) {
    if (max_mx > 256) return cudaErrorInvalidValue;
    if (stage_fits<R, 16>(max_mx, max_my)) return launch_nr<R, 16, true>(a, nsub, (ncols + 15) / 16, max_mx, max_my, st);
    if (stage_fits<R, 8>(max_mx, max_my)) return launch_nr<R, 8, true>(a, nsub, (ncols + 7) / 8, max_mx, max_my, st);
    return launch_nr<R, 4, true>(a, nsub, (ncols + 3) / 4, max_mx, max_my, st);
}

template cudaError_t launch_stage<float>(const StageArgs<float>&, int, int, int, cudaStream_t);
template cudaError_t launch_stage<double>(const StageArgs<double>&, int, int, int, cudaStream_t);
template cudaError_t launch_basis<float>(const StageArgs<float>&, int, int, int, int, cudaStream_t);
template cudaError_t launch_basis<double>(const StageArgs<double>&, int, int, int, int, cudaStream_t);
