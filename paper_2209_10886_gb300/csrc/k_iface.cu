// Interface stages of the sweep schedule: every stage whose local problems
// have zero volume source and whose only output is the outgoing interface
// data (the sweep steps of Sections 4-5 and the residual half-step of the
// block Jacobi update).  For such a stage the local solve followed by the
// trace restriction is the linear map
//
//     u_b = K (cin o G_in),        K = (A_loc^{-1}) restricted to the interface
//                                      boundary points (rows and columns),
//
// and the outgoing data is G_out = ca G_in + cb u_b (the scaled form of
// (-d_{n_{i,j}} - T) u_i, Eq. subPbm), i.e. one application of the paper's
// local scattering operators S_{m(j,i),m(i,k)} of subdomain i (Section 3).
// K is built once per factorisation by batched multi-RHS block solves
// (k_tc.cu / k_stage.cu, basis mode).  One work item (a subdomain, a block of
// RB output rows, a block of NR right-hand sides) gathers the incoming traces,
// runs the GEMV with a warp per output row, applies the transmission and
// scatters the results into the neighbours' slots.  iface_kernel runs one stage
// with one item per CTA; sweep_kernel runs a whole sweep (its stages in order)
// as one cooperative launch, items distributed over the CTAs and a bounded grid
// barrier between stages, so a stage costs a barrier instead of a launch.
#include "helm_internal.cuh"

#include <algorithm>

namespace {

constexpr int IT = 256;      // threads per CTA
constexpr int RB = IFACE_RB; // output rows per work item
constexpr long long SWEEP_WAIT = 2000000000LL;   // cycles (~1 s) before a grid barrier gives up

// LDCG: read through L2 only (data another SM wrote earlier in the same launch)
template <typename T, bool LDCG>
__device__ __forceinline__ T ldg_(const T* p) {
    if (!HELM_CHK(p, sizeof(T))) return T{};
    if constexpr (LDCG) return __ldcg(p);
    else return *p;
}

// mbarrier primitives (the staged form of iface_kernel)
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ bool mb_try(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
// bounded wait (~1 s); false when it expired
__device__ __forceinline__ bool mb_wait(unsigned long long* b, unsigned parity) {
    if (mb_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!mb_try(b, parity))
        if (clock64() - t0 > SWEEP_WAIT) return false;
    return true;
}

// v[s] for a runtime s in 0..3 without indexing the array (keeps it in registers)
__device__ __forceinline__ int sel4(const int (&v)[4], int s) {
    return s == 0 ? v[0] : s == 1 ? v[1] : s == 2 ? v[2] : v[3];
}

// Row stride (elements) of a staged K row: room for a row copied in whole 16-byte
// units from any start, and a multiple of 16 bytes
template <typename T> __host__ __device__ __forceinline__ int staged_ld(int Lb) {
    return sizeof(T) == 8 ? ((Lb + 3) & ~1) : Lb;
}

// One work item of an interface stage: subdomain a.subs[item_sub], output rows
// [row_block*RB, +RB) of its masked sides, the blocks of NR right-hand sides
// rb_first, rb_first + rb_step, ... (the K rows are loaded once for all of them).
// Everything before the gather reads only data that no stage
// writes (the subdomain table and K), so a launch that depends programmatically
// on the previous stage does it while that stage still runs and waits
// (griddepcontrol.wait, a no-op without such a dependency) just before the
// gather.  Staged form (STAGED, one item per CTA): warp 0 first starts
// one bulk copy per output row of K into shared memory (rows at smem_raw,
// staged_ld apart; kofs[q] = where row q starts in its slot).
// the dependency wait of a stage launched after the previous kernel (programmatic
// dependency: griddepcontrol.wait, a no-op without one)
struct GridDepWait {
    __device__ bool operator()() const {
        asm volatile("griddepcontrol.wait;\n" ::: "memory");
        return true;
    }
};

// Returns false when a bounded wait expired (the item was abandoned after its own bulk
// copies completed).  kinit: initialise kbar here (else the caller did, once); kparity:
// the phase of kbar this item's copies complete.  wait(): called by every thread after
// the immutable prologue and before the first read of data earlier stages produce.
// RBI: output rows per item (RB, or fewer for the stage launches of one complex64 RHS)
template <typename R, int NR, bool LDCG, bool STAGED = false, bool MULTI = false, typename WaitF = GridDepWait,
          int RBI = RB>
__device__ bool iface_item(const IfaceArgs<R>& a, int item_sub, int row_block, int rb_first, int rb_step,
                           unsigned char* smem_raw, unsigned long long* kbar = nullptr, int* kofs = nullptr,
                           WaitF wait = WaitF(), bool kinit = true, unsigned kparity = 0) {
    using T = Cx<R>;
    const SubDev sd = HLD(a.subtab + HLD(a.subs + item_sub));
    const int Lb = sd.Lb;
    const int nrb = (a.nrhs + NR - 1) / NR;        // RHS blocks: this item takes rb_first, + rb_step, ...
    // the per-side tables as scalars (a dynamically indexed array would live in local memory)
    const int bo[4] = {sd.bo[0], sd.bo[1], sd.bo[2], sd.bo[3]};
    const int tin[4] = {sd.tin[0], sd.tin[1], sd.tin[2], sd.tin[3]};
    auto len = [&](int s) { return s < 2 ? sd.my : sd.mx; };
    auto on = [&](int s) { return ((a.mask >> s) & 1) && sel4(bo, s) >= 0; };
    // output rows: points of the masked interface sides, in the order W, E, S, N
    int rcount = 0;
#pragma unroll
    for (int s = 0; s < 4; ++s)
        if (on(s)) rcount += len(s);
    const int row0 = row_block * RBI;
    if (row0 >= rcount) return true;
    // side s and point pt of output row `row` (s = -1 past the last row)
    auto locate = [&](int row, int& s, int& pt) {
        s = -1;
        pt = row;
#pragma unroll
        for (int t = 0; t < 4; ++t)
            if (s < 0 && on(t)) {
                if (pt < len(t)) s = t;
                else pt -= len(t);
            }
        if (row >= rcount) s = -1;
    };
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    constexpr bool staged = STAGED;
    const int Lbp = staged_ld<T>(Lb);
    T* Ks = reinterpret_cast<T*>(smem_raw);        // staged: [RBI][Lbp] rows of K
    if (staged && warp == 0) {
        // lane q < RBI copies row row0 + q: from the 16-byte unit holding its first element
        // to the one holding its last (complex64 rows need not start on a unit)
        long long a0 = 0;
        unsigned nbytes = 0;
        if (lane < RBI) {
            int s, pt;
            locate(row0 + lane, s, pt);
            int off = 0;
            if (s >= 0) {
                const long long el = sd.koff + (long long)(sel4(bo, s) + pt) * Lb;
                if constexpr (sizeof(T) == 8) {
                    a0 = el & ~1LL;
                    off = (int)(el - a0);
                    nbytes = (unsigned)((off + Lb + 1) & ~1) * 8u;
                } else {
                    a0 = el;
                    nbytes = (unsigned)Lb * (unsigned)sizeof(T);
                }
            }
            kofs[lane] = off;
        }
        unsigned tot = nbytes;
        for (int o = 16; o > 0; o >>= 1) tot += __shfl_xor_sync(0xffffffffu, tot, o);
        if (lane == 0) {
            if (kinit) {
                asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(kbar)) : "memory");
                asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
            }
            asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(kbar)), "r"(tot)
                         : "memory");
        }
        __syncwarp();
        if (nbytes > 0 && HELM_CHK(a.K + a0, nbytes))     // checking build: a failed check times out the wait
            asm volatile(
                "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
                    smem_u32(Ks + (size_t)lane * Lbp)),
                "l"(a.K + a0), "r"(nbytes), "r"(smem_u32(kbar))
                : "memory");
    }
    // the rows of this warp and their transmission coefficients (immutable: before the wait)
    constexpr int RPW = RBI / (IT / 32);
    static_assert(RPW >= 1 && RPW * (IT / 32) == RBI, "whole rows per warp");
    constexpr int CU = (NR >= 8 || (sizeof(R) == 8 && NR >= 4)) ? 4 : 8;   // fits the register bound
    int srow[RPW], krow[RPW];
    long long tofs[RPW];
    T cca[RPW], ccb[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        int s, pt;
        locate(row0 + warp + q * (IT / 32), s, pt);
        srow[q] = s;
        krow[q] = s >= 0 ? sel4(bo, s) + pt : 0;
        tofs[q] = 0;
        cca[q] = ccb[q] = czero<T>();
        if (s >= 0) {
            const TraceCoef<T> c = HLD(a.tc + sel4(tin, s) + pt);
            cca[q] = c.ca;
            ccb[q] = c.cb;
            tofs[q] = (long long)(s == 0 ? sd.tout[0] : s == 1 ? sd.tout[1] : s == 2 ? sd.tout[2] : sd.tout[3]) + pt;
        }
    }
    // the incoming data, base and sub were written by earlier stages
    if (!wait()) {
        if (staged && warp == 0 && lane == 0) mb_wait(kbar, kparity);   // no copy outlives the item (bounded)
        __syncthreads();
        return false;
    }
    // MULTI = false: exactly one block (straight-line code)
    for (int rb = rb_first; MULTI ? rb < nrb : rb == rb_first; rb += rb_step) {
    const int rhs0 = rb * NR;
    const int nr = min(NR, a.nrhs - rhs0);
    // base - sub of the warp's outputs, loaded alongside the gather: one RHS, lane 0;
    // several, lane k for RHS k (the lane that forms that RHS's outputs)
    T bsub[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        T v = czero<T>();
        const int k = NR == 1 ? 0 : lane;
        if ((NR == 1 ? lane == 0 : lane < nr) && srow[q] >= 0) {
            const long long o = (long long)(rhs0 + k) * a.ntrace + tofs[q];
            if (a.base) v = ldg_<T, LDCG>(a.base + o);
            if (a.sub) v = csub(v, ldg_<T, LDCG>(a.sub + o));
        }
        bsub[q] = v;
    }

    T* graw = staged ? Ks + (size_t)RBI * Lbp : reinterpret_cast<T*>(smem_raw);  // [NR][Lb] incoming data
    T* g = graw + (size_t)NR * Lb;                 // [NR][Lb] cin * incoming data
    if constexpr (NR == 1) {
    // every load of up to GU elements per thread is issued before the first is used
    constexpr int GU = 4;
    for (int i0 = threadIdx.x; i0 < NR * Lb; i0 += IT * GU) {
        T G[GU], C[GU];
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const int idx = i0 + u * IT;
            G[u] = C[u] = czero<T>();
            if (idx < NR * Lb) {
                const int k = idx / Lb, e = idx - k * Lb;
                // the side holding boundary point e: the last interface side starting at or before it
                int s = 0;
#pragma unroll
                for (int q = 1; q < 4; ++q)
                    if (bo[q] >= 0 && e >= bo[q]) s = q;
                const long long ti = sel4(tin, s) + (e - sel4(bo, s));
                if (k < nr) {
                    const long long o = (long long)(rhs0 + k) * a.ntrace + ti;
                    if (a.gin0) G[u] = ldg_<T, LDCG>(a.gin0 + o);
                    if (a.gin1) G[u] = cadd(G[u], ldg_<T, LDCG>(a.gin1 + o));
                    C[u] = HLD(a.tc + ti).cin;
                }
            }
        }
#pragma unroll
        for (int u = 0; u < GU; ++u) {
            const int idx = i0 + u * IT;
            if (idx < NR * Lb) {
                graw[idx] = G[u];
                g[idx] = cmul(G[u], C[u]);
            }
        }
    }
    } else {
    // several RHS: a thread takes boundary points, finds the point's trace index and
    // coefficient once and issues the loads of all the block's RHS together
    for (int e = threadIdx.x; e < Lb; e += IT) {
        int s = 0;
#pragma unroll
        for (int q = 1; q < 4; ++q)
            if (bo[q] >= 0 && e >= bo[q]) s = q;
        const long long ti = sel4(tin, s) + (e - sel4(bo, s));
        const T cin = HLD(a.tc + ti).cin;
        T G[NR];
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            G[k] = czero<T>();
            if (k < nr) {
                const long long o = (long long)(rhs0 + k) * a.ntrace + ti;
                if (a.gin0) G[k] = ldg_<T, LDCG>(a.gin0 + o);
                if (a.gin1) G[k] = cadd(G[k], ldg_<T, LDCG>(a.gin1 + o));
            }
        }
#pragma unroll
        for (int k = 0; k < NR; ++k) {
            graw[k * Lb + e] = G[k];
            g[k * Lb + e] = cmul(G[k], cin);
        }
    }
    }
    if (staged && rb == rb_first) {
        // every thread waits for the copies (bounded); a timeout anywhere ends the item
        __shared__ int kfail;
        if (threadIdx.x == 0) kfail = 0;
        __syncthreads();
        if (!mb_wait(kbar, kparity)) kfail = 1;
        __syncthreads();
        if (kfail) {
            if (threadIdx.x == 0) {
                atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
                mb_wait(kbar, kparity);             // no copy outlives the CTA, bounded again
            }
            return false;
        }
    } else {
        __syncthreads();
    }

    const T* K = a.K + sd.koff;
    // each warp takes RPW rows and keeps the loads of all of them in flight: columns in
    // groups of CU per lane (32 CU per group), every load of a group issued before its FMAs
    const T* Kr[RPW];
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        const int lr = warp + q * (IT / 32);       // row within the item
        if constexpr (STAGED) Kr[q] = Ks + (size_t)lr * Lbp + kofs[lr];
        else Kr[q] = K + (long long)krow[q] * Lb;
    }
    T acc[RPW][NR];
#pragma unroll
    for (int q = 0; q < RPW; ++q)
#pragma unroll
        for (int k = 0; k < NR; ++k) acc[q][k] = czero<T>();
    for (int c0 = lane; c0 < Lb; c0 += 32 * CU) {
        T kv[RPW][CU];
#pragma unroll
        for (int q = 0; q < RPW; ++q)
#pragma unroll
            for (int u = 0; u < CU; ++u) {
                const int c = c0 + 32 * u;
                kv[q][u] = (srow[q] >= 0 && c < Lb) ? (STAGED ? Kr[q][c] : HLD(Kr[q] + c)) : czero<T>();
            }
#pragma unroll
        for (int u = 0; u < CU; ++u) {
            const int c = c0 + 32 * u;
            if (c < Lb) {
#pragma unroll
                for (int k = 0; k < NR; ++k) {
                    const T gv = g[k * Lb + c];
#pragma unroll
                    for (int q = 0; q < RPW; ++q) acc[q][k] = cfma(kv[q][u], gv, acc[q][k]);
                }
            }
        }
    }
#pragma unroll
    for (int q = 0; q < RPW; ++q) {
        if constexpr (NR == 1) {
            for (int o = 16; o > 0; o >>= 1) {
                acc[q][0].x += __shfl_down_sync(0xffffffffu, acc[q][0].x, o);
                acc[q][0].y += __shfl_down_sync(0xffffffffu, acc[q][0].y, o);
            }
            if (lane == 0 && srow[q] >= 0) {
                const T out = cadd(cfma(ccb[q], acc[q][0], cmul(cca[q], graw[krow[q]])), bsub[q]);
                const long long o = (long long)rhs0 * a.ntrace + tofs[q];
                HST(a.dst + o, out);
                if (a.dst2) HST(a.dst2 + o, out);
            }
        } else {
            // butterfly: every lane ends with the row's sums; lane k forms RHS k's output
            T mine = czero<T>();
#pragma unroll
            for (int k = 0; k < NR; ++k) {
                for (int o = 16; o > 0; o >>= 1) {
                    acc[q][k].x += __shfl_xor_sync(0xffffffffu, acc[q][k].x, o);
                    acc[q][k].y += __shfl_xor_sync(0xffffffffu, acc[q][k].y, o);
                }
                if (k == lane) mine = acc[q][k];
            }
            if (lane < nr && srow[q] >= 0) {
                const T out = cadd(cfma(ccb[q], mine, cmul(cca[q], graw[lane * Lb + krow[q]])), bsub[q]);
                const long long o = (long long)(rhs0 + lane) * a.ntrace + tofs[q];
                HST(a.dst + o, out);
                if (a.dst2) HST(a.dst2 + o, out);
            }
        }
    }
    __syncthreads();                                // the shared gather is reused by the next block
    }
    return true;
}

// One stage, one item per CTA, launched with a programmatic dependency on the
// previous kernel of the stream: each CTA lets the next stage launch at once
// (that stage waits for this one to complete before its gather).
// ---------------------------------------------------------------------------
// Dependency-driven persistent sweep: every interface stage of a sweep in one
// cooperative launch, without grid barriers.  The work items (stage, subdomain of
// the stage, block of RB output rows) are dealt to the CTAs in their global order
// (stage-major); an item waits only for the items of earlier stages that write the
// trace slots it reads or touch the slots it writes (a per-(stage, subdomain)
// completion counter, `need` row blocks each), which the host derives from the
// slots' read and write sets.  Meanwhile its K rows are already on their way into
// shared memory.  Waits are bounded (HELM_ERR_TIMEOUT, then the CTA returns after
// its own copies landed).  Deadlock-free with all CTAs resident: a wait points to a
// strictly earlier stage, and each CTA runs its items in order.
struct DepWait {
    const int* deps;           // counter ids this item waits for
    int ndep;
    const int* need;           // per counter id: row-block items that complete it
    const int* counters;
    int* err;
    volatile int* sflag;
    __device__ bool operator()() const {
        if (threadIdx.x == 0) {
            const long long t0 = clock64();
            for (int d = 0; d < ndep && !*sflag; ++d) {
                const int u = deps[d], want = need[u];
                for (;;) {
                    int cur;
                    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(cur) : "l"(counters + u) : "memory");
                    if (cur >= want) break;
                    if (clock64() - t0 > SWEEP_WAIT) {
                        atomicExch(err, (int)HELM_ERR_TIMEOUT);
                        *sflag = 1;
                        break;
                    }
                }
            }
        }
        __syncthreads();
        return *sflag == 0;
    }
};

template <typename R, int NR>
__global__ void __launch_bounds__(IT) sweep_dep_kernel(IfaceArgs<R> base, const SweepStage* stages, const int4* items,
                                                       int nitems, const int* need, const int2* unit_deps,
                                                       const int* deps, int* counters) {
    using T = Cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long kbar;
    __shared__ int kofs[RB];
    __shared__ int sflag;
    if (threadIdx.x == 0) {
        sflag = 0;
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&kbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    T* const* bufs = reinterpret_cast<T* const*>(base.bufs);
    unsigned parity = 0;
    for (int it = blockIdx.x; it < nitems; it += gridDim.x) {
        const int4 d = items[it];                     // stage, subdomain in the stage, row block, counter id
        const SweepStage& st = stages[d.x];
        IfaceArgs<R> a = base;
        a.subs = base.subs + st.sub_off;
        a.gin0 = st.in0 >= 0 ? bufs[st.in0] : nullptr;
        a.gin1 = st.in1 >= 0 ? bufs[st.in1] : nullptr;
        a.mask = st.mask;
        a.dst = st.dst >= 0 ? bufs[st.dst] : nullptr;
        a.dst2 = st.dst2 >= 0 ? bufs[st.dst2] : nullptr;
        a.base = st.base >= 0 ? bufs[st.base] : nullptr;
        a.sub = st.sub >= 0 ? bufs[st.sub] : nullptr;
        const int2 ud = unit_deps[d.w];
        const DepWait w{deps + ud.x, ud.y, need, counters, base.err, &sflag};
        const bool ok =
            iface_item<R, NR, true, true, true, DepWait>(a, d.y, d.z, 0, 1, smem_raw, &kbar, kofs, w, false, parity);
        parity ^= 1u;
        if (!ok) return;
        // publish: the item's stores (ordered before this point by the item's final
        // __syncthreads) precede the count
        if (threadIdx.x == 0) {
            __threadfence();
            atomicAdd(counters + d.w, 1);
        }
    }
}

template <typename R, int NR, bool STAGED, bool MULTI, int RBI>
__global__ void __launch_bounds__(IT) iface_kernel(IfaceArgs<R> a) {
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ __align__(8) unsigned long long kbar;
    __shared__ int kofs[RBI];
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    iface_item<R, NR, false, STAGED, MULTI, GridDepWait, RBI>(a, blockIdx.x, blockIdx.y, blockIdx.z, gridDim.z,
                                                              smem_raw, &kbar, kofs);
}

// grid-wide barrier of a cooperative launch; false (and HELM_ERR_TIMEOUT in err) when it expired
__device__ bool sweep_barrier(unsigned* bar, int* err, volatile int* sflag) {
    // bar[0] counts arrivals, bar[1] is the generation; the last arrival resets the count
    // and publishes the next generation with release semantics, the others poll it with
    // acquire loads (CTA writes before the barrier are ordered by __syncthreads and the
    // release of thread 0's arrival)
    __syncthreads();
    if (threadIdx.x == 0) {
        unsigned g, arrived;
        asm volatile("ld.relaxed.gpu.global.u32 %0, [%1];" : "=r"(g) : "l"(bar + 1) : "memory");
        asm volatile("atom.acq_rel.gpu.global.add.u32 %0, [%1], 1;" : "=r"(arrived) : "l"(bar) : "memory");
        if (arrived == gridDim.x - 1) {
            asm volatile("st.relaxed.gpu.global.u32 [%0], %1;" ::"l"(bar), "r"(0u) : "memory");
            asm volatile("st.release.gpu.global.u32 [%0], %1;" ::"l"(bar + 1), "r"(g + 1) : "memory");
        } else {
            const long long t0 = clock64();
            unsigned cur;
            do {
                asm volatile("ld.acquire.gpu.global.u32 %0, [%1];" : "=r"(cur) : "l"(bar + 1) : "memory");
                if (cur == g && clock64() - t0 > SWEEP_WAIT) {
                    atomicExch(err, (int)HELM_ERR_TIMEOUT);
                    *sflag = 1;
                    break;
                }
            } while (cur == g);
        }
    }
    __syncthreads();
    return *sflag == 0;
}

template <typename R, int NR>
__global__ void __launch_bounds__(IT) sweep_kernel(IfaceArgs<R> base, const SweepStage* stages, int nstages,
                                                   unsigned* bar, int* err) {
    using T = Cx<R>;
    extern __shared__ __align__(16) unsigned char smem_raw[];
    __shared__ int sflag;
    if (threadIdx.x == 0) sflag = 0;
    __syncthreads();
    T* const* bufs = reinterpret_cast<T* const*>(base.bufs);
    const int rblocks = (base.nrhs + NR - 1) / NR;
    for (int s = 0; s < nstages; ++s) {
        const SweepStage& st = stages[s];
        IfaceArgs<R> a = base;
        a.subs = base.subs + st.sub_off;
        a.gin0 = st.in0 >= 0 ? bufs[st.in0] : nullptr;
        a.gin1 = st.in1 >= 0 ? bufs[st.in1] : nullptr;
        a.mask = st.mask;
        a.dst = st.dst >= 0 ? bufs[st.dst] : nullptr;
        a.dst2 = st.dst2 >= 0 ? bufs[st.dst2] : nullptr;
        a.base = st.base >= 0 ? bufs[st.base] : nullptr;
        a.sub = st.sub >= 0 ? bufs[st.sub] : nullptr;
        const int rowb = (st.max_rows + RB - 1) / RB;
        const int items = st.nsub * rowb * rblocks;
        for (int it = blockIdx.x; it < items; it += gridDim.x) {
            const int sub_i = it / (rowb * rblocks);
            const int rem = it - sub_i * rowb * rblocks;
            iface_item<R, NR, true>(a, sub_i, rem / rblocks, rem % rblocks, 1 << 30, smem_raw);
        }
        if (s + 1 < nstages && !sweep_barrier(bar, err, &sflag)) return;
    }
}

template <typename R, int NR, bool STAGED, bool MULTI, int RBI>
cudaError_t launch_nr_s_m(const IfaceArgs<R>& a, int nactive, int max_rows, size_t smem, int zb, cudaStream_t st) {
    cudaError_t e = cudaFuncSetAttribute(iface_kernel<R, NR, STAGED, MULTI, RBI>,
                                         cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(nactive, (max_rows + RBI - 1) / RBI, zb);
    cfg.blockDim = dim3(IT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeProgrammaticStreamSerialization;
    attr[0].val.programmaticStreamSerializationAllowed = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, iface_kernel<R, NR, STAGED, MULTI, RBI>, a);
}

// RHS blocks: each CTA stages its K rows once and loops over the blocks z, z + gridDim.z,
// ...; gridDim.z spreads them only as far as needed for `waves` CTAs per SM
template <typename R, int NR, bool STAGED, int RBI>
cudaError_t launch_nr_s(const IfaceArgs<R>& a, int nactive, int max_rows, size_t smem, int waves, cudaStream_t st) {
    static int sms = 0;
    if (sms == 0) {
        int dev = 0;
        if (cudaGetDevice(&dev) != cudaSuccess ||
            cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
            sms = 1;
    }
    const long long items = (long long)nactive * ((max_rows + RBI - 1) / RBI);
    const int nrb = (a.nrhs + NR - 1) / NR;
    const long long want = (long long)std::max(1, waves) * sms;
    const int zb = (int)std::min<long long>(nrb, std::max<long long>(1, (want + items - 1) / items));
    if (zb == nrb) return launch_nr_s_m<R, NR, STAGED, false, RBI>(a, nactive, max_rows, smem, zb, st);
    return launch_nr_s_m<R, NR, STAGED, true, RBI>(a, nactive, max_rows, smem, zb, st);
}

// staged when allowed, when the item's K rows and gather fit two CTAs per SM and K is
// 16-byte aligned.  One complex64 RHS: items of 8 rows (twice the CTAs of 16-row items,
// one row per warp; measured 23.1 vs 23.5 ms per solve on the 1023^2 workload, where the
// sweep stages give each CTA an SM and its product over the staged rows is bound by
// shared-memory reads); several RHS keep 16 rows (8 measured 3 % slower at 64 RHS)
template <typename R, int NR>
cudaError_t launch_nr(const IfaceArgs<R>& a, int nactive, int max_rows, int max_Lb, int staged_ok, int waves,
                      cudaStream_t st) {
    using T = Cx<R>;
    constexpr int RBI = (sizeof(R) == 4 && NR == 1) ? RB / 2 : RB;
    const size_t gather = 2 * (size_t)NR * max_Lb * sizeof(T);
    const size_t staged = (size_t)RBI * staged_ld<T>(max_Lb) * sizeof(T) + gather;
    if (staged_ok && staged <= 113 * 1024 && (reinterpret_cast<uintptr_t>(a.K) & 15) == 0)
        return launch_nr_s<R, NR, true, RBI>(a, nactive, max_rows, staged, waves, st);
    return launch_nr_s<R, NR, false, RBI>(a, nactive, max_rows, gather, waves, st);
}

template <typename R, int NR>
cudaError_t launch_sweep_nr(const IfaceArgs<R>& a, const SweepStage* stages, int nstages, int max_Lb, int grid,
                            unsigned* bar, int* err, cudaStream_t st) {
    using T = Cx<R>;
    size_t smem = 2 * (size_t)NR * max_Lb * sizeof(T);
    cudaError_t e = cudaFuncSetAttribute(sweep_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    IfaceArgs<R> aa = a;
    void* args[] = {&aa, (void*)&stages, &nstages, &bar, &err};
    count_launch();
    return cudaLaunchCooperativeKernel((const void*)sweep_kernel<R, NR>, dim3(grid), dim3(IT), args, smem, st);
}

template <typename R, int NR>
cudaError_t launch_sweep_dep_nr(const IfaceArgs<R>& a, const SweepStage* stages, const int4* items, int nitems,
                                const int* need, const int2* unit_deps, const int* deps, int* counters, int max_Lb,
                                cudaStream_t st) {
    using T = Cx<R>;
    const size_t smem = (size_t)RB * staged_ld<T>(max_Lb) * sizeof(T) + 2 * (size_t)NR * max_Lb * sizeof(T);
    if (smem > 227 * 1024 || (reinterpret_cast<uintptr_t>(a.K) & 15) != 0) return cudaErrorNotSupported;
    cudaError_t e = cudaFuncSetAttribute(sweep_dep_kernel<R, NR>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    int dev = 0, sms = 0, per = 0;
    if ((e = cudaGetDevice(&dev)) != cudaSuccess) return e;
    if ((e = cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev)) != cudaSuccess) return e;
    if ((e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep_dep_kernel<R, NR>, IT, smem)) != cudaSuccess)
        return e;
    if (per < 1) return cudaErrorNotSupported;
    const int grid = (int)std::min<long long>((long long)std::min(per, 2) * sms, nitems);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(std::max(grid, 1));
    cfg.blockDim = dim3(IT);
    cfg.dynamicSmemBytes = smem;
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    count_launch();
    return cudaLaunchKernelEx(&cfg, sweep_dep_kernel<R, NR>, a, stages, items, nitems, need, unit_deps, deps, counters);
}

}  // namespace

// CTAs of the sweep kernel that are co-resident on the device (0: cooperative launch unavailable)
template <typename R>
int sweep_grid(int nrhs, int max_Lb) {
    int dev = 0, sms = 0, coop = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev) != cudaSuccess || !coop) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    const size_t smem = 2 * (size_t)(nrhs >= 4 ? 4 : nrhs >= 2 ? 2 : 1) * max_Lb * sizeof(Cx<R>);
    cudaError_t e;
    if (nrhs >= 4) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep_kernel<R, 4>, IT, smem);
    else if (nrhs >= 2) e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep_kernel<R, 2>, IT, smem);
    else e = cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, sweep_kernel<R, 1>, IT, smem);
    if (e != cudaSuccess || per < 1) return 0;
    return sms;                       // one CTA per SM: the grid barrier costs one arrival per CTA
}

template <typename R>
cudaError_t launch_sweep(const IfaceArgs<R>& a, const SweepStage* stages, int nstages, int max_Lb, int grid,
                         unsigned* bar, int* err, cudaStream_t st) {
    if (nstages == 0 || a.nrhs == 0) return cudaSuccess;
    if (grid <= 0) return cudaErrorNotSupported;
    if (a.nrhs >= 4) return launch_sweep_nr<R, 4>(a, stages, nstages, max_Lb, grid, bar, err, st);
    if (a.nrhs >= 2) return launch_sweep_nr<R, 2>(a, stages, nstages, max_Lb, grid, bar, err, st);
    return launch_sweep_nr<R, 1>(a, stages, nstages, max_Lb, grid, bar, err, st);
}

// the interface stages of a sweep as one dependency-driven cooperative launch (see
// sweep_dep_kernel); counters must be zero on entry
template <typename R>
cudaError_t launch_sweep_dep(const IfaceArgs<R>& a, const SweepStage* stages, const int4* items, int nitems,
                             const int* need, const int2* unit_deps, const int* deps, int* counters, int max_Lb,
                             cudaStream_t st) {
    if (nitems == 0 || a.nrhs == 0) return cudaSuccess;
    if (a.nrhs >= 4) return launch_sweep_dep_nr<R, 4>(a, stages, items, nitems, need, unit_deps, deps, counters, max_Lb, st);
    if (a.nrhs >= 2) return launch_sweep_dep_nr<R, 2>(a, stages, items, nitems, need, unit_deps, deps, counters, max_Lb, st);
    return launch_sweep_dep_nr<R, 1>(a, stages, items, nitems, need, unit_deps, deps, counters, max_Lb, st);
}

template <typename R>
cudaError_t launch_iface(const IfaceArgs<R>& a, int nactive, int max_rows, int max_Lb, cudaStream_t st,
                         const IfaceCfg* cfg) {
    if (nactive == 0 || a.nrhs == 0) return cudaSuccess;
    // default: blocks of 4 RHS (at 64 RHS on the 1023^2 workload, 16 measured 2x slower
    // when every block had its own CTA); the autotuner may pick another shape
    if constexpr (sizeof(R) == 4)
        if (cfg && cfg->tc) {
            // the tensor-core form walks all boundary points of its rows in one CTA: only a
            // stage with at least two of its CTAs per SM (by default) keeps every SM's tensor
            // pipe busy
            static int sms = 0;
            if (sms == 0) {
                int dev = 0;
                if (cudaGetDevice(&dev) != cudaSuccess ||
                    cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess)
                    sms = 1;
            }
            const long long ctas = (long long)nactive * ((max_rows + 127) / 128) * ((a.nrhs + cfg->tc_nb - 1) / cfg->tc_nb);
            if (ctas >= (cfg->tc_min_ctas >= 0 ? (long long)cfg->tc_min_ctas : 2LL * sms))
                return launch_iface_tc(a, nactive, max_rows, cfg->tc, cfg->tc_nb, 2 * sms, max_Lb, st);
        }
    const int nr = cfg ? cfg->nr : (a.nrhs >= 4 ? 4 : a.nrhs >= 2 ? 2 : 1);
    const int staged_ok = cfg ? cfg->staged : 1;
    const int waves = cfg ? cfg->waves : 3;
    if constexpr (sizeof(R) == 4)   // complex128 blocks of 16 would spill
        if (nr >= 16) return launch_nr<R, 16>(a, nactive, max_rows, max_Lb, staged_ok, waves, st);
    if (nr >= 8) return launch_nr<R, 8>(a, nactive, max_rows, max_Lb, staged_ok, waves, st);
    if (nr >= 4) return launch_nr<R, 4>(a, nactive, max_rows, max_Lb, staged_ok, waves, st);
    if (nr >= 2) return launch_nr<R, 2>(a, nactive, max_rows, max_Lb, staged_ok, waves, st);
    return launch_nr<R, 1>(a, nactive, max_rows, max_Lb, staged_ok, waves, st);
}

template cudaError_t launch_iface<float>(const IfaceArgs<float>&, int, int, int, cudaStream_t, const IfaceCfg*);
template cudaError_t launch_iface<double>(const IfaceArgs<double>&, int, int, int, cudaStream_t, const IfaceCfg*);
template cudaError_t launch_sweep_dep<float>(const IfaceArgs<float>&, const SweepStage*, const int4*, int, const int*,
                                             const int2*, const int*, int*, int, cudaStream_t);
template cudaError_t launch_sweep_dep<double>(const IfaceArgs<double>&, const SweepStage*, const int4*, int, const int*,
                                              const int2*, const int*, int*, int, cudaStream_t);
template int sweep_grid<float>(int, int);
template int sweep_grid<double>(int, int);
template cudaError_t launch_sweep<float>(const IfaceArgs<float>&, const SweepStage*, int, int, int, unsigned*, int*,
                                         cudaStream_t);
template cudaError_t launch_sweep<double>(const IfaceArgs<double>&, const SweepStage*, int, int, int, unsigned*, int*,
                                          cudaStream_t);
