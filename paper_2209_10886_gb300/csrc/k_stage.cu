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
// row-major storage: consumer threads own output columns (row groups split
// the rows of each chunk), coalesced rows in shared memory.  X is stored as
// two column halves (each half row-major, see SubDev), streamed from HBM by
// bulk (TMA) copies that one producer thread issues into a ring of shared
// memory slots guarded by full/empty mbarriers.
//
// A subdomain is solved either by one CTA (both halves) or by a cluster of
// two CTAs, one per half: each computes its half of y, and after every grid
// row the two exchange their halves of the next input vector through
// distributed shared memory (st.async stores counted as bytes on the
// receiver's mbarrier).  Every
// wait is bounded in time; on expiry the kernel records HELM_ERR_TIMEOUT in a
// device flag, finishes its (now meaningless) steps without waiting, drains
// its own copies and skips the epilogue.
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
// the same with acquire semantics at cluster scope (data written by the peer CTA)
__device__ __forceinline__ bool mbar_try_cluster(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.acquire.cluster.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_addr(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// wait for the phase with this parity, at most `limit` cycles
template <bool CLUSTER>
__device__ __forceinline__ bool mbar_wait(unsigned long long* b, unsigned parity, long long limit) {
    auto t = [&]() { return CLUSTER ? mbar_try_cluster(b, parity) : mbar_try(b, parity); };
    if (t()) return true;
    const long long t0 = clock64();
    while (!t())
        if (clock64() - t0 > limit) return false;
    return true;
}
__device__ __forceinline__ void bulk_copy(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    if (!HELM_CHK(src, bytes)) return;                  // checking build: the wait then gives up
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_addr(dst)),
        "l"(src), "r"(bytes), "r"(smem_addr(bar))
        : "memory");
}
__device__ __forceinline__ void consumer_sync(int nthreads) {
    asm volatile("bar.sync 1, %0;\n" ::"r"(nthreads) : "memory");
}
// address of the same shared-memory location in CTA `rank` of the cluster
__device__ __forceinline__ unsigned peer_addr(const void* p, unsigned rank) {
    unsigned r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;\n" : "=r"(r) : "r"(smem_addr(p)), "r"(rank));
    return r;
}
// store into the peer CTA's shared memory, counted as complete_tx bytes on the peer's
// mbarrier `bar` (the completion releases the data at cluster scope)
__device__ __forceinline__ void st_async_peer(unsigned addr, float2 v, unsigned bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f32 [%0], {%1, %2}, [%3];\n" ::"r"(addr),
                 "f"(v.x), "f"(v.y), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void st_async_peer(unsigned addr, double2 v, unsigned bar) {
    asm volatile("st.async.shared::cluster.mbarrier::complete_tx::bytes.v2.f64 [%0], {%1, %2}, [%3];\n" ::"r"(addr),
                 "d"(v.x), "d"(v.y), "r"(bar)
                 : "memory");
}
__device__ __forceinline__ void cluster_sync_all() {
    asm volatile("barrier.cluster.arrive.aligned;\nbarrier.cluster.wait.aligned;\n" ::: "memory");
}

// BASIS = true: the NR right-hand sides of a CTA are unit data at consecutive
// interface boundary points (columns of the boundary operator K, see StageArgs).
// csize = 1: one CTA per subdomain; csize = 2: a cluster of two, one per column half.
template <typename R, int NR, bool BASIS>
__global__ void __launch_bounds__(NR <= 4 ? 544 : 288) stage_kernel(StageArgs<R> a, int rows_per_chunk, int nslots,
                                                                  int cwarps, int ngroups, int csize) {
    using T = Cx<R>;
    extern __shared__ __align__(128) unsigned char smem_raw[];
    // xbar[b]: the peer's half of the next v of the steps with step & 1 == b (cluster form)
    __shared__ __align__(8) unsigned long long full_bar[MAXNS], empty_bar[MAXNS], xbar[2];
    __shared__ int abort_flag;

    const int rank = csize == 2 ? (int)(blockIdx.x & 1) : 0;
    const int s = BASIS ? blockIdx.x / csize : HLD(a.subs + blockIdx.x / csize);
    const SubDev sd = HLD(a.subtab + s);
    const int mx = sd.mx, my = sd.my;
    const int rhs0 = blockIdx.y * NR;                    // first RHS (workspace slot) of this CTA
    const int e0 = BASIS ? a.col0 + rhs0 : 0;            // first boundary point (basis mode)
    // uniform across the cluster: both CTAs share blockIdx.y and the subdomain
    if (BASIS && e0 >= sd.Lb) return;
    const int nr = BASIS ? min(NR, sd.Lb - e0) : min(NR, a.nrhs - rhs0);
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    // columns of this CTA: the half `rank` (cluster) or all of them
    const int w0 = sd.w0;
    const int c_lo = csize == 2 ? (rank ? w0 : 0) : 0;
    const int c_hi = csize == 2 ? (rank ? mx : w0) : mx;
    const int peer_cols = rank ? w0 : mx - w0;           // columns the peer CTA owns (cluster form)
    // consumers: ngroups groups of cwarps warps; thread (grp, c) sums the rows
    // grp, grp + ngroups, ... of every chunk for output column c_lo + c
    const int ncons = 32 * cwarps * ngroups;
    const bool producer = warp == cwarps * ngroups;
    const int col = c_lo + tid % (32 * cwarps);
    const int grp = tid / (32 * cwarps);
    const bool worker = !producer && col < c_hi;
    const bool owner = worker && grp == 0;               // finishes column col of every row
    const int myhalf = col < w0 ? 0 : 1;
    const int Rch = rows_per_chunk;
    const int nq = (mx + Rch - 1) / Rch;                 // chunks per half per step
    const int h_first = csize == 2 ? rank : 0;           // halves streamed by this CTA
    const int nhalves = csize == 2 ? 1 : (w0 < mx ? 2 : 1);   // a one-node-wide subdomain has one half
    const int cps = nq * nhalves;                        // chunks per step
    const int nsteps = 2 * my - 1;
    const int Q = nsteps * cps;
    const int mxp = 32 * ((mx + 31) / 32 > 0 ? (mx + 31) / 32 : 1);   // v rows (full length)
    const int cw = 32 * cwarps;                                        // part rows (this CTA's columns)
    // boundary arrays per RHS: W[my] | E[my] | S[mx] | N[mx]
    const int L = 2 * (mx + my);
    auto boff = [&](int side) { return side < 2 ? side * my : 2 * my + (side - 2) * mx; };
    const int ldh[2] = {sd.ld0, sd.ld1};
    const long long hoff1 = (long long)mx * sd.ld0;     // element offset of half 1 in X_r
    const long long xr_elems = (long long)mx * (sd.ld0 + sd.ld1);
    const int ldmax = max(sd.ld0, sd.ld1);

    // dynamic shared memory: ring[nslots][Rch*ldmax] | v[2][NR][mxp_max] | binc[NR][L] | ub[NR][L] | part
    T* ring = reinterpret_cast<T*>(smem_raw);
    const size_t slot_elems = (size_t)Rch * ldmax;
    T* vbuf = ring + (size_t)nslots * slot_elems;
    T* binc = vbuf + 2 * (size_t)NR * mxp;
    T* ub = binc + (size_t)NR * L;
    T* part = ub + (size_t)NR * L;                       // [ngroups-1][NR][cw] row-group partial sums

    const long long N = (long long)a.nx * a.ny;
    const T* Xs = a.X + sd.xoff;

    auto gin = [&](int k, long long idx) -> T {
        T g = a.gin0 ? HLD(a.gin0 + (long long)(rhs0 + k) * a.ntrace + idx) : czero<T>();
        if (a.gin1) g = cadd(g, HLD(a.gin1 + (long long)(rhs0 + k) * a.ntrace + idx));
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
        return HLD(a.r + (long long)(rhs0 + k) * N + (long long)(sd.y0 + r) * a.nx + sd.x0 + c);
    };
    double rsc[NR], zsc[NR];
#pragma unroll
    for (int k = 0; k < NR; ++k) {
        rsc[k] = (a.rscale && k < nr) ? HLD(a.rscale + rhs0 + k) : 1.0;
        zsc[k] = (a.zscale && k < nr) ? HLD(a.zscale + rhs0 + k) : 1.0;
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
            HST(a.z + (long long)(rhs0 + k) * N + (long long)(sd.y0 + r) * a.nx + sd.x0 + c,
                make_double2(zu.x * zsc[k], zu.y * zsc[k]));
        }
    };
    // is boundary point e (of side `side`, index pt along it) in this CTA's columns?
    auto owns_point = [&](int side, int pt) {
        const int c = side == SW ? 0 : side == SE ? mx - 1 : pt;
        return c >= c_lo && c < c_hi;
    };

    // ---- prologue: barriers, incoming terms G_in/(1-beta) into shared memory, v = b_1
    if (tid == 0) {
        for (int i = 0; i < nslots; ++i) {
            mbar_init(&full_bar[i], 1);
            mbar_init(&empty_bar[i], cwarps * ngroups);
        }
        mbar_init(&xbar[0], 1);
        mbar_init(&xbar[1], 1);
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
            b = cmul(gin(k, ti), HLD(a.tc + ti).cin);
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
    // both CTAs of a cluster have initialised their barriers before any remote arrival
    if (csize == 2) cluster_sync_all();

    if (producer) {
        // ---- producer: one thread streams the chunks of X_1..X_my, X_{my-1}..X_1
        if (lane == 0) {
            int r = 0, q = 0, hh = 0, slot = 0, step = 0;
            unsigned ph = 0;
            int issued = 0;
            for (int t = 0; t < Q; ++t) {
                if (*((volatile int*)&abort_flag)) break;
                if (t >= nslots && !mbar_wait<false>(&empty_bar[slot], ph ^ 1u, WAIT_LIMIT)) {
                    abort_flag = 1;
                    if (a.err) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
                    break;
                }
                const int half = h_first + hh;
                const int ld = ldh[half];
                const int rows = min(Rch, mx - q * Rch);
                const unsigned bytes = (unsigned)((size_t)rows * ld * sizeof(T));
                const T* src = Xs + (long long)r * xr_elems + (half ? hoff1 : 0) + (long long)q * Rch * ld;
                mbar_expect_tx(&full_bar[slot], bytes);
                bulk_copy(ring + (size_t)slot * slot_elems, src, bytes, &full_bar[slot]);
                ++issued;
                if (++slot == nslots) { slot = 0; ph ^= 1u; }
                if (++q == nq) {
                    q = 0;
                    if (++hh == nhalves) {
                        hh = 0;
                        ++step;
                        r = step < my ? step : 2 * my - 2 - step;
                    }
                }
            }
            if (*((volatile int*)&abort_flag)) {
                // drain: wait (bounded) for every copy this CTA issued before leaving
                for (int t = max(0, issued - nslots); t < issued; ++t)
                    mbar_wait<false>(&full_bar[t % nslots], (unsigned)((t / nslots) & 1), WAIT_LIMIT);
            }
        }
    } else {
        // ---- consumers: y = X v column-wise
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
            for (int c = 0; c < cps; ++c) {
                const int half = h_first + c / nq, q = c % nq;
                const bool ab = *((volatile int*)&abort_flag) != 0;
                if (!mbar_wait<false>(&full_bar[slot], ph, ab ? 0 : WAIT_LIMIT)) {
                    abort_flag = 1;
                    if (a.err) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
                }
                if (worker && half == myhalf && !*((volatile int*)&abort_flag)) {
                    const int ld = ldh[half];
                    const T* S = ring + (size_t)slot * slot_elems + (col - (half ? w0 : 0));
                    const T* vq = v + q * Rch;
                    const int rows = min(Rch, mx - q * Rch);
                    const int G = ngroups;
                    int jj = grp;
                    for (; jj + 3 * G < rows; jj += 4 * G) {
                        const T x0 = S[(size_t)(jj + 0 * G) * ld], x1 = S[(size_t)(jj + 1 * G) * ld];
                        const T x2 = S[(size_t)(jj + 2 * G) * ld], x3 = S[(size_t)(jj + 3 * G) * ld];
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
                        const T x0 = S[(size_t)jj * ld];
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
                        part[((size_t)(grp - 1) * NR + k) * cw + (col - c_lo)] = sum;
                    }
                }
                consumer_sync(ncons);
                if (owner) {
#pragma unroll
                    for (int k = 0; k < NR; ++k)
                        for (int g2 = 1; g2 < ngroups; ++g2)
                            acc[k][0] = cadd(acc[k][0], part[((size_t)(g2 - 1) * NR + k) * cw + (col - c_lo)]);
                }
            }
            const bool last = step == nsteps - 1;
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
                            HST(ywk + (long long)r * mx + col, sum);              // y_r
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
                        if (r >= 1) ynext[k] = HLD(ywk + (long long)(r - 1) * mx + col);
                    }
                    vn[k * mxp + col] = nv;
                    if (csize == 2 && !last)
                        st_async_peer(peer_addr(&vn[k * mxp + col], rank ^ 1), nv, peer_addr(&xbar[step & 1], rank ^ 1));
                }
            }
            consumer_sync(ncons);
            if (csize == 2 && !last) {
                // exchange: my half of the next v went to the peer by st.async; the peer's
                // half arrives the same way, counted as bytes on xbar[step & 1] (each barrier
                // completes every other step, so a half of step s + 2 cannot count towards
                // step s)
                if (tid == 0) mbar_expect_tx(&xbar[step & 1], (unsigned)(peer_cols * nr * sizeof(T)));
                const bool ab = *((volatile int*)&abort_flag) != 0;
                if (!mbar_wait<true>(&xbar[step & 1], (unsigned)((step >> 1) & 1), ab ? 1000 : WAIT_LIMIT)) {
                    abort_flag = 1;
                    if (a.err) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
                }
            }
            cur ^= 1;
        }
    }
    // no CTA of a cluster leaves while its peer may still write into its shared memory
    if (csize == 2) cluster_sync_all();
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
            if (!owns_point(side, pt)) continue;
            HST(a.K + sd.koff + (long long)(e0 + k) * sd.Lb + sd.bo[side] + pt, ub[idx]);
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
            if (!owns_point(side, pt)) continue;
            const long long in = sd.tin[side] + pt, out = sd.tout[side] + pt;
            const TraceCoef<T> c = HLD(a.tc + in);
            T g = cfma(c.cb, ub[idx], cmul(c.ca, gin(k, in)));
            const long long o = (long long)(rhs0 + k) * a.ntrace + out;
            if (a.base) g = cadd(g, HLD(a.base + o));
            if (a.sub) g = csub(g, HLD(a.sub + o));
            HST(a.dst + o, g);
            if (a.dst2) HST(a.dst2 + o, g);
        }
    }
}

// Launch geometry of one stage launch.
struct Geo {
    int csize, cwarps, ngroups, rows, nslots;
    size_t smem;
};

// chunk_kb > 0: that chunk size only (the autotuner's choice), else the rule below
template <typename R, int NR>
static bool geometry(int max_mx, int max_my, int max_w, int max_ld, int csize, Geo& g, int chunk_kb = 0) {
    using T = Cx<R>;
    g.csize = csize;
    const int width = csize == 2 ? max_w : max_mx;       // columns of one CTA
    g.cwarps = (width + 31) / 32;
    g.ngroups = NR <= 4 ? std::max(1, std::min(8, 16 / g.cwarps)) : 1;
    const int mxp = 32 * ((max_mx + 31) / 32);
    const size_t fixed = 2 * (size_t)NR * mxp * sizeof(T) + 2 * (size_t)NR * 2 * (max_mx + max_my) * sizeof(T) +
                         (size_t)(g.ngroups - 1) * NR * 32 * g.cwarps * sizeof(T);
    const size_t budget = 227 * 1024 - 1024;
    if (fixed >= budget) return false;
    // the largest chunk (64, 48 or 32 KB, a multiple of 4 rows) that leaves three ring
    // slots: the copy engine streams few large copies faster than many small ones
    int rows = 0, nslots = 0;
    const int kbs[3] = {chunk_kb > 0 ? chunk_kb : 64, chunk_kb > 0 ? chunk_kb : 48, chunk_kb > 0 ? chunk_kb : 32};
    for (int kb : kbs) {
        rows = (int)((size_t)kb * 1024 / ((size_t)max_ld * sizeof(T)));
        rows = std::min(std::max(4, rows & ~3), max_mx);
        nslots = std::min((int)((budget - fixed) / ((size_t)rows * max_ld * sizeof(T))), MAXNS);
        if (nslots >= 3) break;
    }
    if (nslots < 2) return false;
    g.rows = rows;
    g.nslots = nslots;
    g.smem = fixed + (size_t)nslots * rows * max_ld * sizeof(T);
    return true;
}

template <typename R, int NR, bool BASIS>
cudaError_t launch_nr(const StageArgs<R>& a, int nunits, int ny_blocks, const Geo& g, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(stage_kernel<R, NR, BASIS>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                         (int)g.smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nunits * g.csize, ny_blocks);
    cfg.blockDim = dim3(32 * (g.cwarps * g.ngroups + 1));
    cfg.dynamicSmemBytes = g.smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeClusterDimension;
    attr[0].val.clusterDim.x = g.csize;
    attr[0].val.clusterDim.y = 1;
    attr[0].val.clusterDim.z = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, stage_kernel<R, NR, BASIS>, a, g.rows, g.nslots, g.cwarps, g.ngroups, g.csize);
}

}  // namespace

template <typename R>
cudaError_t launch_stage(const StageArgs<R>& a, int nactive, int max_mx, int max_my, int max_w, int max_ld,
                         int num_sms, cudaStream_t st, const StageCfg* cfg) {
    if (nactive == 0) return cudaSuccess;
    if (max_mx > 256) return cudaErrorInvalidValue;
    // two CTAs per subdomain when the stage leaves enough SMs idle: one SM alone streams a
    // subdomain's factors well below its share of HBM (complex64) or is bound by its FP64
    // units (complex128); the autotuner may choose otherwise
    int csize = (2 * nactive * std::max(1, (a.nrhs + 15) / 16) <= num_sms && max_mx >= 64) ? 2 : 1;
    if (cfg && cfg->csize > 0) csize = cfg->csize;
    const int kb = cfg ? cfg->chunk_kb : 0;
    Geo g;
#define HELM_TRY_NR(NRV)                                                                                    \
    if (a.nrhs >= NRV && geometry<R, NRV>(max_mx, max_my, max_w, max_ld, csize, g, kb))                    \
        return launch_nr<R, NRV, false>(a, nactive, (a.nrhs + NRV - 1) / NRV, g, st);
    HELM_TRY_NR(16)
    HELM_TRY_NR(8)
    HELM_TRY_NR(4)
    HELM_TRY_NR(2)
#undef HELM_TRY_NR
    if (!geometry<R, 1>(max_mx, max_my, max_w, max_ld, csize, g, kb)) return cudaErrorInvalidValue;
    return launch_nr<R, 1, false>(a, nactive, a.nrhs, g, st);
}

template <typename R>
cudaError_t launch_basis(const StageArgs<R>& a, int nsub, int ncols, int max_mx, int max_my, int max_w, int max_ld,
                         cudaStream_t st) {
    if (max_mx > 256) return cudaErrorInvalidValue;
    Geo g;
    if (geometry<R, 16>(max_mx, max_my, max_w, max_ld, 1, g)) return launch_nr<R, 16, true>(a, nsub, (ncols + 15) / 16, g, st);
    if (geometry<R, 8>(max_mx, max_my, max_w, max_ld, 1, g)) return launch_nr<R, 8, true>(a, nsub, (ncols + 7) / 8, g, st);
    if (geometry<R, 4>(max_mx, max_my, max_w, max_ld, 1, g)) return launch_nr<R, 4, true>(a, nsub, (ncols + 3) / 4, g, st);
    return cudaErrorInvalidValue;
}

template cudaError_t launch_stage<float>(const StageArgs<float>&, int, int, int, int, int, int, cudaStream_t,
                                        const StageCfg*);
template cudaError_t launch_stage<double>(const StageArgs<double>&, int, int, int, int, int, int, cudaStream_t,
                                         const StageCfg*);
template cudaError_t launch_basis<float>(const StageArgs<float>&, int, int, int, int, int, int, cudaStream_t);
template cudaError_t launch_basis<double>(const StageArgs<double>&, int, int, int, int, int, int, cudaStream_t);
