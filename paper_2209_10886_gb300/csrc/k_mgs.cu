// Modified Gram-Schmidt step of the FP64 Arnoldi process in one persistent,
// cooperatively launched kernel.
//
// For every right-hand side: w <- w - sum_k h_k v_k with h_k = v_k^H w taken
// against the current w (modified Gram-Schmidt: 4 FP64 FMA per element for the
// dot and 4 for the update of each basis vector, half of classical
// Gram-Schmidt with reorthogonalisation), then h_{j+1,j} = ||w|| and
// v_{j+1} = w / ||w||.  Each CTA keeps its slice of w in registers for the
// whole process; each projection reads its slice of v_k once from HBM (the
// update re-reads it from L1).  The dot products are reduced deterministically:
// every CTA writes its partial sum, passes a grid barrier, and adds all
// partials in the same order.  Barrier waits are bounded in time; on expiry the
// kernel records HELM_ERR_TIMEOUT and returns.  When two slices of the vector per
// CTA fit in shared memory, mgs_smem_kernel streams the basis vectors there by
// bulk copies issued one step ahead.
#include <algorithm>

#include "helm_internal.cuh"

namespace {

constexpr int MT = 256;                          // threads per CTA
constexpr long long BAR_LIMIT = 2000000000LL;    // cycles (~1 s): the default limit of a grid barrier

struct MgsArgs {
    const double2* V;          // basis: v_k of RHS r at V + k*vsk + r*vsr
    long long vsk, vsr;
    double2* w;                // new vector of RHS r at w + r*vsr (overwritten by v_{j+1})
    int nvec;                  // j + 1 basis vectors to project out
    long long n;
    int nrhs;
    const int* active;
    double2* hcol;             // h_k of RHS r at hcol[r*ldh + k]
    int ldh;
    double* hnorm;             // ||w|| after the projections, per RHS
    double2* partial;          // [2 * gridDim.x] scratch of partial sums
    unsigned* bar;             // [0] arrival count, [1] generation (zero before the first launch)
    int* err;
    long long limit;           // cycles a grid barrier waits before it gives up
};

__device__ __forceinline__ double2 warp_sum2(double2 v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

// grid-wide barrier over co-resident CTAs; returns false when the wait expired
__device__ bool grid_barrier(unsigned* bar, int* err, int* sflag, long long limit) {
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
                if (cur == g && clock64() - t0 > limit) {
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

// sum of the gridDim.x partials in a fixed order, broadcast to the CTA
__device__ double2 sum_partials(const double2* partial, double2* sh) {
    double2 t = make_double2(0.0, 0.0);
    if (threadIdx.x < 32) {
        for (int c = threadIdx.x; c < (int)gridDim.x; c += 32) {
            const double2 v = HLDCG(partial + c);
            t.x += v.x;
            t.y += v.y;
        }
        t = warp_sum2(t);
        if (threadIdx.x == 0) sh[0] = t;
    }
    __syncthreads();
    t = sh[0];
    __syncthreads();
    return t;
}

// block sum of a complex value into partial[blockIdx.x] (sh holds 1 + blockDim.x / 32 values)
__device__ void block_partial(double2 v, double2* partial, double2* sh) {
    v = warp_sum2(v);
    const int wid = threadIdx.x >> 5, lane = threadIdx.x & 31;
    if (lane == 0) sh[1 + wid] = v;
    __syncthreads();
    if (threadIdx.x == 0) {
        double2 t = make_double2(0.0, 0.0);
        for (int i = 0; i < (int)(blockDim.x >> 5); ++i) { t.x += sh[1 + i].x; t.y += sh[1 + i].y; }
        partial[blockIdx.x] = t;
    }
}

template <int EPT>
__global__ void __launch_bounds__(MT) mgs_kernel(MgsArgs a) {
    __shared__ double2 sh[1 + MT / 32];
    __shared__ int sflag;
    if (threadIdx.x == 0) sflag = 0;
    __syncthreads();
    const long long stride = (long long)gridDim.x * MT;
    const long long base = (long long)blockIdx.x * MT + threadIdx.x;
    // reduction s writes partial[(s & 1) * gridDim.x + cta]: a CTA can only write
    // reduction s+1 after every CTA has passed barrier s, i.e. has read reduction
    // s-1 (which used the other half), so one barrier per reduction suffices
    unsigned s = 0;
    auto reduce = [&](double2 v, double2& out) -> bool {
        double2* part = a.partial + (s & 1u) * gridDim.x;
        block_partial(v, part, sh);
        if (!grid_barrier(a.bar, a.err, &sflag, a.limit)) return false;
        out = sum_partials(part, sh);
        ++s;
        return true;
    };
    for (int r = 0; r < a.nrhs; ++r) {
        if (a.active && !a.active[r]) continue;
        double2* w = a.w + r * a.vsr;
        double2 wr[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const long long p = base + e * stride;
            wr[e] = p < a.n ? HLD(w + p) : make_double2(0.0, 0.0);
        }
        // step k: finish the update with v_{k-1} (h_{k-1} known) and, in the same
        // pass over the elements, the dot product with v_k against the updated w
        double2 mh = make_double2(0.0, 0.0);
        const double2* vprev = nullptr;
        for (int k = 0; k < a.nvec; ++k) {
            const double2* v = a.V + k * a.vsk + r * a.vsr;
            // four independent partial sums: short FP64 dependency chains
            double2 acc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const long long p = base + e * stride;
                if (p < a.n) {
                    if (vprev) wr[e] = cfma(mh, HLD(vprev + p), wr[e]);
                    acc[e & 3] = cfmaconj(HLD(v + p), wr[e], acc[e & 3]);
                }
            }
            const double2 accs = make_double2((acc[0].x + acc[1].x) + (acc[2].x + acc[3].x),
                                              (acc[0].y + acc[1].y) + (acc[2].y + acc[3].y));
            double2 h;
            if (!reduce(accs, h)) return;
            if (blockIdx.x == 0 && threadIdx.x == 0) HST(a.hcol + (long long)r * a.ldh + k, h);
            mh = make_double2(-h.x, -h.y);
            vprev = v;
        }
        double nrm = 0.0;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const long long p = base + e * stride;
            if (vprev && p < a.n) wr[e] = cfma(mh, HLD(vprev + p), wr[e]);
            nrm = fma(wr[e].x, wr[e].x, fma(wr[e].y, wr[e].y, nrm));
        }
        double2 tot;
        if (!reduce(make_double2(nrm, 0.0), tot)) return;
        const double hn = sqrt(tot.x);
        if (blockIdx.x == 0 && threadIdx.x == 0) HST(a.hnorm + r, hn);
        const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const long long p = base + e * stride;
            if (p < a.n) HST(w + p, make_double2(wr[e].x * inv, wr[e].y * inv));
        }
    }
}

// ---------------------------------------------------------------------------
// The same process with the basis streamed through shared memory: CTA b owns the
// contiguous elements [b*L, b*L + L); v_{k+1} is fetched by one bulk (TMA) copy
// while the grid reduces h_k, so no memory latency follows a barrier.  Buffer
// k & 1 holds v_k; the pass of step k reads v_{k-1} (update) and v_k (dot), after
// which v_{k+1} is copied into the buffer v_{k-1} occupied.
__device__ __forceinline__ unsigned smem_u32(const void* p) { return (unsigned)__cvta_generic_to_shared(p); }
__device__ __forceinline__ void mb_init(unsigned long long* b) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(b)) : "memory");
}
__device__ __forceinline__ bool mb_try(unsigned long long* b, unsigned parity) {
    unsigned ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok)
        : "r"(smem_u32(b)), "r"(parity)
        : "memory");
    return ok != 0;
}
__device__ __forceinline__ bool mb_wait(unsigned long long* b, unsigned parity) {
    if (mb_try(b, parity)) return true;
    const long long t0 = clock64();
    while (!mb_try(b, parity))
        if (clock64() - t0 > BAR_LIMIT) return false;
    return true;
}
// one thread: copy `bytes` (a multiple of 16, both addresses 16-byte aligned) into shared memory
__device__ __forceinline__ void bulk_fetch(void* dst, const void* src, unsigned bytes, unsigned long long* bar) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;\n" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
    if (!HELM_CHK(src, bytes)) return;                  // checking build: the wait then gives up
    asm volatile(
        "cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];\n" ::"r"(
            smem_u32(dst)),
        "l"(src), "r"(bytes), "r"(smem_u32(bar))
        : "memory");
}

template <int EPT, int NT>
__global__ void __launch_bounds__(NT) mgs_smem_kernel(MgsArgs a, int L) {
    extern __shared__ __align__(16) double2 vbuf[];           // [2][L]
    __shared__ double2 sh[1 + NT / 32];
    __shared__ __align__(8) unsigned long long full[2];
    __shared__ int sflag;
    const long long c0 = (long long)blockIdx.x * L;
    const int len = (int)max(0LL, min((long long)L, a.n - c0));   // elements of this CTA
    if (threadIdx.x == 0) {
        sflag = 0;
        mb_init(&full[0]);
        mb_init(&full[1]);
        asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    }
    __syncthreads();
    unsigned fills[2] = {0u, 0u};                             // completed fills per buffer (for the parity)
    unsigned s = 0;
    auto reduce = [&](double2 v, double2& out) -> bool {
        double2* part = a.partial + (s & 1u) * gridDim.x;
        block_partial(v, part, sh);
        if (!grid_barrier(a.bar, a.err, &sflag, a.limit)) return false;
        out = sum_partials(part, sh);
        ++s;
        return true;
    };
    auto fetch = [&](const double2* v, int b) {
        if (threadIdx.x == 0 && len > 0) bulk_fetch(vbuf + (size_t)b * L, v + c0, (unsigned)len * 16u, &full[b]);
    };
    auto wait_buf = [&](int b) -> bool {
        if (len == 0) return true;
        const bool ok = mb_wait(&full[b], fills[b] & 1u);
        ++fills[b];
        if (!ok) {
            if (threadIdx.x == 0) atomicExch(a.err, (int)HELM_ERR_TIMEOUT);
            return false;
        }
        return true;
    };
    for (int r = 0; r < a.nrhs; ++r) {
        if (a.active && !a.active[r]) continue;
        double2* w = a.w + r * a.vsr;
        double2 wr[EPT];
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int i = e * NT + threadIdx.x;
            wr[e] = i < len ? HLD(w + c0 + i) : make_double2(0.0, 0.0);
        }
        const double2* V = a.V + r * a.vsr;
        __syncthreads();                                       // the buffers are free
        fetch(V, 0);
        double2 mh = make_double2(0.0, 0.0);
        for (int k = 0; k < a.nvec; ++k) {
            const int b = k & 1;
            if (!wait_buf(b)) return;                          // every thread times out the same way
            const double2* vk = vbuf + (size_t)b * L;
            const double2* vp = vbuf + (size_t)(b ^ 1) * L;
            double2 acc[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) acc[q] = make_double2(0.0, 0.0);
#pragma unroll
            for (int e = 0; e < EPT; ++e) {
                const int i = e * NT + threadIdx.x;
                if (i < len) {
                    if (k > 0) wr[e] = cfma(mh, vp[i], wr[e]);
                    acc[e & 3] = cfmaconj(vk[i], wr[e], acc[e & 3]);
                }
            }
            const double2 accs = make_double2((acc[0].x + acc[1].x) + (acc[2].x + acc[3].x),
                                              (acc[0].y + acc[1].y) + (acc[2].y + acc[3].y));
            __syncthreads();                                   // v_{k-1} is no longer read
            if (k + 1 < a.nvec) fetch(V + (long long)(k + 1) * a.vsk, b ^ 1);
            double2 h;
            if (!reduce(accs, h)) {
                if (k + 1 < a.nvec) wait_buf(b ^ 1);          // no copy outlives the CTA
                return;
            }
            if (blockIdx.x == 0 && threadIdx.x == 0) HST(a.hcol + (long long)r * a.ldh + k, h);
            mh = make_double2(-h.x, -h.y);
        }
        const double2* vl = vbuf + (size_t)((a.nvec - 1) & 1) * L;
        double nrm0 = 0.0, nrm1 = 0.0;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int i = e * NT + threadIdx.x;
            if (i < len) {
                if (a.nvec > 0) wr[e] = cfma(mh, vl[i], wr[e]);
                if (e & 1) nrm1 = fma(wr[e].x, wr[e].x, fma(wr[e].y, wr[e].y, nrm1));
                else nrm0 = fma(wr[e].x, wr[e].x, fma(wr[e].y, wr[e].y, nrm0));
            }
        }
        double2 tot;
        if (!reduce(make_double2(nrm0 + nrm1, 0.0), tot)) return;
        const double hn = sqrt(tot.x);
        if (blockIdx.x == 0 && threadIdx.x == 0) HST(a.hnorm + r, hn);
        const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
#pragma unroll
        for (int e = 0; e < EPT; ++e) {
            const int i = e * NT + threadIdx.x;
            if (i < len) HST(w + c0 + i, make_double2(wr[e].x * inv, wr[e].y * inv));
        }
    }
}

template <int EPT, int NT>
cudaError_t launch_smem_ept(MgsArgs& a, int grid, int L, cudaStream_t st) {
    const size_t smem = 2 * (size_t)L * sizeof(double2);
    cudaError_t e =
        cudaFuncSetAttribute(mgs_smem_kernel<EPT, NT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    if (e != cudaSuccess) return e;
    void* args[] = {&a, &L};
    count_launch();
    return cudaLaunchCooperativeKernel((const void*)mgs_smem_kernel<EPT, NT>, dim3(grid), dim3(NT), args, smem, st);
}

template <int EPT>
cudaError_t launch_ept(MgsArgs& a, int grid, cudaStream_t st) {
    void* args[] = {&a};
    count_launch();
    return cudaLaunchCooperativeKernel((const void*)mgs_kernel<EPT>, dim3(grid), dim3(MT), args, 0, st);
}

// ---------------------------------------------------------------------------
// Classical Gram-Schmidt with selective reorthogonalisation (the DGKS test: a
// second pass when ||w'||^2 < eta2 ||w||^2, eta2 = 1/2 by default) for short vectors, one cooperative
// launch per Arnoldi step: CTA b keeps the contiguous slice [b*L, b*L + L) of w
// in shared memory; a pass computes all j+1 dot products (warp q takes the basis
// vectors q + 16 t and q + 8 + 16 t), reduces them over the grid (one barrier),
// and updates its slice against the basis read from L2.  The norm, the
// normalisation of v_{j+1} and the Givens update of the least-squares problem
// (CTA 0) follow in the same launch.  VT = double2 or float2: products, updates
// and the Givens arithmetic in the vectors' precision; sums across CTAs, the
// coefficients and the stored least-squares problem in FP64 (the serial chain of
// rotations in FP64 costs ~0.6 us per rotation on GB300's narrow FP64 pipe).  Reductions are deterministic: every CTA adds
// the partials of all CTAs in the same order, so every CTA takes the same branches.
// ||w'||^2 comes from ||w||^2 - ||h||^2 (no reduction of its own) when that keeps at
// least 2 eta2 of ||w||^2.  1 grid barrier per RHS then, 2 when ||w'||^2 is reduced,
// 4 when the second pass runs, each bounded in time (HELM_ERR_TIMEOUT, then return).
template <typename VT>
struct Cgs2Args {
    const VT* V;               // basis: v_k of RHS r at V + k*vsk + r*vsr; w = v_{j+1} in place
    long long vsk, vsr;
    int j;                     // new column j: j+1 basis vectors to project out
    long long n;
    int nrhs;
    const int* active;
    double2* hsum;             // h_{0..j,j} of RHS r at hsum[r*ldh + k] (both passes summed)
    int ldh;
    double* hnorm;             // h_{j+1,j} per RHS
    int* need;                 // 1 where the second pass ran
    // Arnoldi least-squares state (the Hessenberg step)
    double2* H;                // column-major per RHS, H(i, jj) at H[r*hs + jj*ldH + i]
    int ldH;
    long long hs;
    double2 *cs, *sn, *g;      // rotations and rotated right-hand side, ldg per RHS
    int ldg;
    double* est;               // |g_{j+1}| per RHS
    double* invh;              // 1 / h_{j+1,j}
    double2* partial;          // [2][gridDim.x][j + 2] scratch
    unsigned* bar;
    int* err;
    int L;                     // slice length per CTA
    const int* dj;             // when set, j is read from here (a device-driven loop)
    const VT* wsrc;            // when set, w = -wsrc (RHS r at wsrc + r*vsr) instead of the slot j + 1
    VT* vout1;                 // when set, v_{j+1} is also written here and to vout2 (RHS r at + r*vsr)
    VT* vout2;
    long long limit;           // cycles a grid barrier waits before it gives up
    double eta2;               // second pass when ||w'||^2 < eta2 ||w||^2
};

constexpr int CT = 256;        // threads per CTA of the fused step

template <typename VT> __device__ __forceinline__ VT warp_sumc(VT v) {
    for (int o = 16; o > 0; o >>= 1) {
        v.x += __shfl_down_sync(0xffffffffu, v.x, o);
        v.y += __shfl_down_sync(0xffffffffu, v.y, o);
    }
    return v;
}

template <typename VT>
__global__ void __launch_bounds__(CT, 1) cgs2_step_kernel(Cgs2Args<VT> a) {
    // the next kernel (the loop control) may launch now; it waits for this one to complete
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int J = a.dj ? *a.dj : a.j;             // the new column
    using Re = decltype(VT::x);
    extern __shared__ __align__(16) double2 csm[];
    double2* hv = csm;                              // [j + 2] reduced values of the current pass
    double2* h1 = hv + (J + 2);                   // [j + 1] coefficients, both passes
    double2* gv = h1 + (J + 1);                   // [3 (j + 2)] Givens scratch (CTA 0)
    VT* hc = reinterpret_cast<VT*>(gv + 3 * (J + 2));   // [j + 1] -hv in the vectors' precision
    VT* ws = hc + (J + 1);                        // [L] slice of w
    __shared__ double red[CT / 32];
    __shared__ double2 gsum[CT];                    // group sums of the grid reduction
    __shared__ int sflag;
    const int nvec = J + 1, PS = J + 2;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const long long c0 = (long long)blockIdx.x * a.L;
    const int len = (int)max(0LL, min((long long)a.L, a.n - c0));
    if (threadIdx.x == 0) sflag = 0;
    __syncthreads();
    unsigned s = 0;
    // CTA sum of one value per thread (all threads see it after the call)
    auto block_sum = [&](double v) -> double {
        for (int o = 16; o > 0; o >>= 1) v += __shfl_down_sync(0xffffffffu, v, o);
        __syncthreads();
        if (lane == 0) red[warp] = v;
        __syncthreads();
        double t = 0.0;
        for (int q = 0; q < CT / 32; ++q) t += red[q];
        return t;
    };
    // partials of this CTA are in part[cta*PS + 0..cnt); after the barrier every CTA
    // sums column k over all CTAs in the same order into hv[k].  Per block of up to
    // 32 columns: KP (a power of two >= the block's columns) lanes per column set,
    // thread t takes column t % KP and the CTAs t / KP, t / KP + CT / KP, ... (loads
    // coalesced along k, few per thread); a butterfly over the lanes of equal column,
    // then the CT / 32 warp sums in order
    auto grid_reduce = [&](double2* part, int cnt) -> bool {
        if (!grid_barrier(a.bar, a.err, &sflag, a.limit)) return false;
        const int G = (int)gridDim.x;
        for (int kb = 0; kb < cnt; kb += 32) {
            const int rem = min(32, cnt - kb);
            int KP = 1;
            while (KP < rem) KP <<= 1;
            const int groups = CT / KP;
            const int kq = threadIdx.x & (KP - 1), grp = threadIdx.x / KP;
            double2 t = make_double2(0.0, 0.0);
            if (kq < rem) {
                for (int c0 = grp; c0 < G; c0 += groups * 8) {
                    double2 pv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int c = c0 + groups * u;
                        pv[u] = c < G ? HLDCG(part + (long long)c * PS + kb + kq) : make_double2(0.0, 0.0);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) { t.x += pv[u].x; t.y += pv[u].y; }
                }
            }
            for (int o = 16; o >= KP; o >>= 1) {
                t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
                t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
            }
            if (lane < KP) gsum[warp * KP + lane] = t;
            __syncthreads();
            if (threadIdx.x < rem) {
                double2 v = gsum[threadIdx.x];
                for (int q = 1; q < CT / 32; ++q) { v.x += gsum[q * KP + threadIdx.x].x; v.y += gsum[q * KP + threadIdx.x].y; }
                hv[kb + threadIdx.x] = v;
            }
            __syncthreads();
        }
        ++s;
        return true;
    };
    auto cur_part = [&]() { return a.partial + (size_t)(s & 1u) * gridDim.x * PS; };
    // dot products of the slice with all basis vectors into this CTA's partials, 8
    // elements of two vectors per lane loaded before they are used
    auto dots = [&](const VT* V, double2* part) {
        for (int ka = warp; ka < nvec; ka += 2 * (CT / 32)) {
            const int kb = ka + CT / 32;
            const bool hb = kb < nvec;
            const VT* va = V + ka * a.vsk + c0;
            const VT* vb = V + (hb ? kb : ka) * a.vsk + c0;
            VT acca = czero<VT>(), accb = acca;
            for (int i0 = 0; i0 < len; i0 += 256) {
                VT xa[8], xb[8];
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + lane + 32 * u;
                    const bool in = i < len;
                    xa[u] = in ? HLDCG(va + i) : czero<VT>();
                    xb[u] = (in && hb) ? HLDCG(vb + i) : czero<VT>();
                }
#pragma unroll
                for (int u = 0; u < 8; ++u) {
                    const int i = i0 + lane + 32 * u;
                    if (i < len) {
                        const VT wv = ws[i];
                        acca = cfmaconj(xa[u], wv, acca);
                        accb = cfmaconj(xb[u], wv, accb);
                    }
                }
            }
            acca = warp_sumc(acca);
            accb = warp_sumc(accb);
            if (lane == 0) {
                part[(long long)blockIdx.x * PS + ka] = make_double2((double)acca.x, (double)acca.y);
                if (hb) part[(long long)blockIdx.x * PS + kb] = make_double2((double)accb.x, (double)accb.y);
            }
        }
    };
    // hc = -hv rounded to the vectors' precision (then a barrier before use)
    auto set_coef = [&]() {
        for (int k = threadIdx.x; k < nvec; k += CT) hc[k] = mk((Re)-hv[k].x, (Re)-hv[k].y);
        __syncthreads();
    };
    // ws += sum_k hc[k] v_k over the slice, 16 basis values per element loaded before
    // they are used; returns this thread's share of ||ws||^2
    auto update = [&](const VT* V) -> double {
        Re nrm = 0;
        for (int i = threadIdx.x; i < len; i += CT) {
            VT x = ws[i];
            const VT* v = V + c0 + i;
            for (int k0 = 0; k0 < nvec; k0 += 16) {
                VT vv[16];
#pragma unroll
                for (int u = 0; u < 16; ++u) vv[u] = k0 + u < nvec ? HLDCG(v + (k0 + u) * a.vsk) : czero<VT>();
#pragma unroll
                for (int u = 0; u < 16; ++u)
                    if (k0 + u < nvec) x = cfma(hc[k0 + u], vv[u], x);
            }
            ws[i] = x;
            nrm = fma(x.x, x.x, fma(x.y, x.y, nrm));
        }
        return (double)nrm;
    };

    for (int r = 0; r < a.nrhs; ++r) {
        if (a.active && !a.active[r]) continue;
        const VT* V = a.V + r * a.vsr;
        VT* w = const_cast<VT*>(V) + (long long)nvec * a.vsk;
        const VT* wsrc = a.wsrc ? a.wsrc + r * a.vsr : nullptr;
        Re n0 = 0;
        for (int i = threadIdx.x; i < len; i += CT) {
            VT x;
            if (wsrc) {
                x = HLD(wsrc + c0 + i);
                x = mk(-x.x, -x.y);
            } else {
                x = HLD(w + c0 + i);
            }
            ws[i] = x;
            n0 = fma(x.x, x.x, fma(x.y, x.y, n0));
        }
        const double w2l = block_sum((double)n0);    // syncs: the slice is in place
        // pass 1: h1 = V^H w and ||w||^2 (column j + 1 of the partials)
        double2* part = cur_part();
        dots(V, part);
        if (threadIdx.x == 0) part[(long long)blockIdx.x * PS + nvec] = make_double2(w2l, 0.0);
        if (!grid_reduce(part, nvec + 1)) return;
        const double w2 = hv[nvec].x;
        // ||h||^2: the same sum, in the same order, in every thread of every CTA
        double hh = 0.0;
        for (int k = 0; k < nvec; ++k) hh = fma(hv[k].x, hv[k].x, fma(hv[k].y, hv[k].y, hh));
        for (int k = threadIdx.x; k < nvec; k += CT) h1[k] = hv[k];
        set_coef();
        const double n1 = block_sum(update(V));
        double hn2;                                  // ||w'||^2
        if (w2 - hh >= 2.0 * a.eta2 * w2) {
            // the projection removed at most 1 - 2 eta2 of ||w||^2: ||w'||^2 = ||w||^2 - ||h||^2
            // loses at most a factor 1 / (2 eta2) of the sums' relative accuracy, and no
            // second pass follows, so the grid reduction of ||w'||^2 is not needed
            hn2 = w2 - hh;
        } else {
            part = cur_part();
            if (threadIdx.x == 0) part[(long long)blockIdx.x * PS] = make_double2(n1, 0.0);
            if (!grid_reduce(part, 1)) return;
            hn2 = hv[0].x;
        }
        const bool second = hn2 < a.eta2 * w2;
        if (second) {
            part = cur_part();
            dots(V, part);
            if (!grid_reduce(part, nvec)) return;
            for (int k = threadIdx.x; k < nvec; k += CT) h1[k] = cadd(h1[k], hv[k]);
            set_coef();
            const double n2 = block_sum(update(V));
            part = cur_part();
            if (threadIdx.x == 0) part[(long long)blockIdx.x * PS] = make_double2(n2, 0.0);
            if (!grid_reduce(part, 1)) return;
            hn2 = hv[0].x;
        }
        const double hn = sqrt(hn2);
        const double inv = hn > 0.0 ? 1.0 / hn : 0.0;
        const Re invr = (Re)inv;
        for (int i = threadIdx.x; i < len; i += CT) {
            const VT v = mk(ws[i].x * invr, ws[i].y * invr);
            HST(w + c0 + i, v);
            if (a.vout1) HST(a.vout1 + r * a.vsr + c0 + i, v);
            if (a.vout2) HST(a.vout2 + r * a.vsr + c0 + i, v);
        }
        if (blockIdx.x == 0) {
            // h column, then the Givens update of the least-squares problem in the
            // vectors' precision: operands converted in parallel, the serial chain on
            // thread 0, the results converted back in parallel
            using C2 = VT;
            C2* col = reinterpret_cast<C2*>(gv);
            C2* csv = col + (J + 2);
            C2* snv = csv + (J + 2);
            double2* csr = a.cs + (long long)r * a.ldg;
            double2* snr = a.sn + (long long)r * a.ldg;
            double2* gr = a.g + (long long)r * a.ldg;
            for (int k = threadIdx.x; k <= J + 1; k += CT) {
                if (k <= J) HST(a.hsum + (long long)r * a.ldh + k, h1[k]);
                const double2 hk = k <= J ? h1[k] : make_double2(hn, 0.0);
                col[k] = mk((Re)hk.x, (Re)hk.y);
                if (k < J) {
                    const double2 ck = HLD(csr + k), sk = HLD(snr + k);
                    csv[k] = mk((Re)ck.x, (Re)0);
                    snv[k] = mk((Re)sk.x, (Re)sk.y);
                }
            }
            __shared__ C2 gpair[2];
            if (threadIdx.x == 0) gpair[0] = mk((Re)HLD(gr + J).x, (Re)HLD(gr + J).y);
            __syncthreads();
            if (threadIdx.x == 0) {
                HST(a.hnorm + r, hn);
                HST(a.need + r, second ? 1 : 0);
                C2 gj = gpair[0], gj1;
                givens_column<C2>(col, csv, snv, J, gj, gj1);
                gpair[0] = gj;
                gpair[1] = gj1;
                HST(a.invh + r, inv);
            }
            __syncthreads();
            double2* colg = a.H + r * a.hs + (long long)J * a.ldH;
            for (int k = threadIdx.x; k <= J + 1; k += CT) HST(colg + k, make_double2((double)col[k].x, (double)col[k].y));
            if (threadIdx.x == 32) {
                HST(csr + J, make_double2((double)csv[J].x, 0.0));
                HST(snr + J, make_double2((double)snv[J].x, (double)snv[J].y));
            }
            if (threadIdx.x == 64) {
                const C2 g0 = gpair[0], g1 = gpair[1];
                HST(gr + J, make_double2((double)g0.x, (double)g0.y));
                HST(gr + J + 1, make_double2((double)g1.x, (double)g1.y));
                HST(a.est + r, sqrt((double)g1.x * (double)g1.x + (double)g1.y * (double)g1.y));
            }
        }
        __syncthreads();                              // ws, hv, hc and h1 are reused by the next RHS
    }
}

// ---------------------------------------------------------------------------
// The same step for several RHS at once (nrhs >= 2): groups of up to CG_MAX RHS go
// through every phase together, so a group costs the grid barriers one RHS does (1, 2
// when any of its RHS needs ||w'||^2 reduced, 4 when any needs the second pass).  The dot products of all (RHS, basis
// vector) pairs of the group and the squared norms (the dot of w with itself) share
// one grid reduction; the second-pass test is per RHS; the Givens updates of the
// group's RHS run on different CTAs.
constexpr int CG_MAX = 16;

template <typename VT>
__global__ void __launch_bounds__(CT, 1) cgs2_group_kernel(Cgs2Args<VT> a, int G) {
    using Re = decltype(VT::x);
    asm volatile("griddepcontrol.launch_dependents;\n" ::: "memory");
    const int J = a.dj ? *a.dj : a.j;               // the new column
    const int nvec = J + 1, PS = J + 2, CS = G * PS;
    extern __shared__ __align__(16) double2 csm[];
    double2* hv = csm;                              // [G * PS] reduced values of the current pass
    double2* h1 = hv + (size_t)G * PS;              // [G * nvec] coefficients, both passes
    double2* gv = h1 + (size_t)G * nvec;            // [3 (J + 2)] Givens scratch
    VT* hc = reinterpret_cast<VT*>(gv + 3 * (J + 2));   // [G * nvec] -hv in the vectors' precision
    VT* ws = hc + (size_t)G * nvec;                 // [G * L] slices of w
    __shared__ double2 gsum[CT];
    __shared__ int sflag;
    __shared__ int gact[CG_MAX], gsec[CG_MAX];
    __shared__ double gw2[CG_MAX], gn2[CG_MAX];
    __shared__ Re ginv[CG_MAX];
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int L = a.L;
    const long long c0 = (long long)blockIdx.x * L;
    const int len = (int)max(0LL, min((long long)L, a.n - c0));
    if (threadIdx.x == 0) sflag = 0;
    __syncthreads();
    unsigned s = 0;
    auto cur_part = [&]() { return a.partial + (size_t)(s & 1u) * gridDim.x * CS; };
    // every CTA adds column k < cnt of all CTAs' partials (stride CS) in the same order
    // into hv[k]: lane = column, warps over CTA groups, a butterfly, the warp sums in order
    auto grid_reduce = [&](double2* part, int cnt) -> bool {
        if (!grid_barrier(a.bar, a.err, &sflag, a.limit)) return false;
        const int Gd = (int)gridDim.x;
        for (int kb = 0; kb < cnt; kb += 32) {
            const int rem = min(32, cnt - kb);
            int KP = 1;
            while (KP < rem) KP <<= 1;
            const int groups = CT / KP;
            const int kq = threadIdx.x & (KP - 1), grp = threadIdx.x / KP;
            double2 t = make_double2(0.0, 0.0);
            if (kq < rem) {
                for (int cb = grp; cb < Gd; cb += groups * 8) {
                    double2 pv[8];
#pragma unroll
                    for (int u = 0; u < 8; ++u) {
                        const int c = cb + groups * u;
                        pv[u] = c < Gd ? HLDCG(part + (long long)c * CS + kb + kq) : make_double2(0.0, 0.0);
                    }
#pragma unroll
                    for (int u = 0; u < 8; ++u) { t.x += pv[u].x; t.y += pv[u].y; }
                }
            }
            for (int o = 16; o >= KP; o >>= 1) {
                t.x += __shfl_xor_sync(0xffffffffu, t.x, o);
                t.y += __shfl_xor_sync(0xffffffffu, t.y, o);
            }
            if (lane < KP) gsum[warp * KP + lane] = t;
            __syncthreads();
            if (threadIdx.x < rem) {
                double2 v = gsum[threadIdx.x];
                for (int q = 1; q < CT / 32; ++q) { v.x += gsum[q * KP + threadIdx.x].x; v.y += gsum[q * KP + threadIdx.x].y; }
                hv[kb + threadIdx.x] = v;
            }
            __syncthreads();
        }
        ++s;
        return true;
    };

    for (int g0 = 0; g0 < a.nrhs; g0 += G) {
        const int gn = min(G, a.nrhs - g0);
        if (threadIdx.x < CG_MAX) {
            const int t = threadIdx.x;
            gact[t] = t < gn && (!a.active || a.active[g0 + t]);
            gsec[t] = 0;
        }
        __syncthreads();
        int any = 0;
        for (int g = 0; g < gn; ++g) any |= gact[g];
        if (!any) continue;                          // every thread reads the same flags
        // partial dots over the slices, one warp per (RHS, vector) pair, PP pairs of a warp
        // with all their loads in flight: mode 0 every basis vector and w itself (the
        // squared norm, k = nvec), mode 1 only w itself (partial at g), mode 2 the basis
        // vectors of the RHS that need a second pass
        constexpr int PP = 4;
        auto dots = [&](int mode, double2* part) {
            const int per = mode == 1 ? 1 : (mode == 0 ? nvec + 1 : nvec);
            const int np = gn * per;
            for (int pb = warp * PP; pb < np; pb += PP * (CT / 32)) {
                const VT* vp[PP];
                const VT* wp[PP];
                bool onp[PP], selfp[PP];          // selfp: w with itself (shared memory, plain loads)
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    const int pr = min(pb + q, np - 1);
                    const int g = pr / per, kk = pr - g * per;
                    const int k = mode == 1 ? nvec : kk;
                    onp[q] = pb + q < np && gact[g] && (mode != 2 || gsec[g]);
                    selfp[q] = k == nvec;
                    wp[q] = ws + (size_t)g * L;
                    vp[q] = k == nvec ? wp[q] : a.V + (long long)k * a.vsk + (long long)(g0 + g) * a.vsr + c0;
                }
                VT acc[PP];
#pragma unroll
                for (int q = 0; q < PP; ++q) acc[q] = czero<VT>();
                for (int i0 = 0; i0 < len; i0 += 256) {
                    VT x[PP][8];
#pragma unroll
                    for (int q = 0; q < PP; ++q)
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int i = i0 + lane + 32 * u;
                            x[q][u] = (onp[q] && i < len) ? (selfp[q] ? wp[q][i] : HLDCG(vp[q] + i)) : czero<VT>();
                        }
#pragma unroll
                    for (int q = 0; q < PP; ++q)
#pragma unroll
                        for (int u = 0; u < 8; ++u) {
                            const int i = i0 + lane + 32 * u;
                            if (i < len) acc[q] = cfmaconj(x[q][u], wp[q][i], acc[q]);
                        }
                }
#pragma unroll
                for (int q = 0; q < PP; ++q) {
                    const VT t = warp_sumc(acc[q]);
                    const int pr = pb + q;
                    if (lane == 0 && pr < np) {
                        const int g = pr / per, kk = pr - g * per;
                        part[(long long)blockIdx.x * CS + (mode == 1 ? g : g * PS + (mode == 1 ? nvec : kk))] =
                            make_double2((double)t.x, (double)t.y);
                    }
                }
            }
        };
        // ws_g += sum_k hc_gk v_k over the slices (mode 0: active RHS, 2: second-pass ones),
        // two elements per thread with all 2 x 16 loads in flight
        auto update = [&](int mode) {
            const int tot = gn * len;
            for (int idx0 = threadIdx.x; idx0 < tot; idx0 += 2 * CT) {
                int gq[2], iq[2];
                bool onq[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) {
                    const int idx = min(idx0 + q * CT, tot - 1);
                    gq[q] = idx / len;
                    iq[q] = idx - gq[q] * len;
                    onq[q] = idx0 + q * CT < tot && gact[gq[q]] && (mode != 2 || gsec[gq[q]]);
                }
                VT xq[2];
#pragma unroll
                for (int q = 0; q < 2; ++q) xq[q] = onq[q] ? ws[(size_t)gq[q] * L + iq[q]] : czero<VT>();
                for (int k0 = 0; k0 < nvec; k0 += 16) {
                    VT vv[2][16];
#pragma unroll
                    for (int q = 0; q < 2; ++q)
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            vv[q][u] = (onq[q] && k0 + u < nvec)
                                           ? HLDCG(a.V + (long long)(k0 + u) * a.vsk + (long long)(g0 + gq[q]) * a.vsr + c0 + iq[q])
                                           : czero<VT>();
#pragma unroll
                    for (int q = 0; q < 2; ++q)
#pragma unroll
                        for (int u = 0; u < 16; ++u)
                            if (k0 + u < nvec) xq[q] = cfma(hc[(size_t)gq[q] * nvec + k0 + u], vv[q][u], xq[q]);
                }
#pragma unroll
                for (int q = 0; q < 2; ++q)
                    if (onq[q]) ws[(size_t)gq[q] * L + iq[q]] = xq[q];
            }
        };
        // the slices of w (the operator's output, negated, when it comes from wsrc)
        for (int idx = threadIdx.x; idx < gn * len; idx += CT) {
            const int g = idx / len, i = idx - g * len;
            if (!gact[g]) continue;
            const long long off = (long long)(g0 + g) * a.vsr + c0 + i;
            VT x;
            if (a.wsrc) {
                x = a.wsrc[off];
                x = mk(-x.x, -x.y);
            } else {
                x = a.V[off + (long long)nvec * a.vsk];
            }
            ws[(size_t)g * L + i] = x;
        }
        __syncthreads();
        double2* part = cur_part();
        dots(0, part);
        if (!grid_reduce(part, gn * PS)) return;
        if (threadIdx.x < gn) gw2[threadIdx.x] = hv[threadIdx.x * PS + nvec].x;
        for (int idx = threadIdx.x; idx < gn * nvec; idx += CT) {
            const int g = idx / nvec, k = idx - g * nvec;
            const double2 h = hv[g * PS + k];
            h1[idx] = h;
            hc[idx] = mk((Re)-h.x, (Re)-h.y);
        }
        __syncthreads();
        update(0);
        // ||w'||^2 = ||w||^2 - ||h||^2 per RHS where the difference keeps at least 2 eta2
        // of ||w||^2 (as in the one-RHS step); a grid reduction of ||w'||^2 otherwise
        if (threadIdx.x < gn) {
            const int g = threadIdx.x;
            double hh = 0.0;
            for (int k = 0; k < nvec; ++k) {
                const double2 h = h1[g * nvec + k];
                hh = fma(h.x, h.x, fma(h.y, h.y, hh));
            }
            gn2[g] = gw2[g] - hh;
            gsec[g] = gact[g] && !(gn2[g] >= 2.0 * a.eta2 * gw2[g]);    // 1: exact norm wanted
        }
        __syncthreads();
        int exact = 0;
        for (int g = 0; g < gn; ++g) exact |= gsec[g];
        if (exact) {
            part = cur_part();
            dots(1, part);
            if (!grid_reduce(part, gn)) return;
            if (threadIdx.x < gn) gn2[threadIdx.x] = hv[threadIdx.x].x;
        }
        __syncthreads();
        if (threadIdx.x < gn) {
            const int g = threadIdx.x;
            gsec[g] = gact[g] && gn2[g] < a.eta2 * gw2[g];
        }
        __syncthreads();
        int anysec = 0;
        for (int g = 0; g < gn; ++g) anysec |= gsec[g];
        if (anysec) {
            part = cur_part();
            dots(2, part);
            if (!grid_reduce(part, gn * PS)) return;
            for (int idx = threadIdx.x; idx < gn * nvec; idx += CT) {
                const int g = idx / nvec, k = idx - g * nvec;
                if (!gsec[g]) continue;
                const double2 h = hv[g * PS + k];
                h1[idx] = cadd(h1[idx], h);
                hc[idx] = mk((Re)-h.x, (Re)-h.y);
            }
            __syncthreads();
            update(2);
            __syncthreads();
            part = cur_part();
            dots(1, part);
            if (!grid_reduce(part, gn)) return;
            if (threadIdx.x < gn && gsec[threadIdx.x]) gn2[threadIdx.x] = hv[threadIdx.x].x;
            __syncthreads();
        }
        if (threadIdx.x < gn) {
            const double hn = sqrt(gn2[threadIdx.x]);
            ginv[threadIdx.x] = (Re)(hn > 0.0 ? 1.0 / hn : 0.0);
        }
        __syncthreads();
        for (int idx = threadIdx.x; idx < gn * len; idx += CT) {
            const int g = idx / len, i = idx - g * len;
            if (!gact[g]) continue;
            const VT x = ws[(size_t)g * L + i];
            const VT v = mk(x.x * ginv[g], x.y * ginv[g]);
            const long long off = (long long)(g0 + g) * a.vsr + c0 + i;
            const_cast<VT*>(a.V)[off + (long long)nvec * a.vsk] = v;
            if (a.vout1) a.vout1[off] = v;
            if (a.vout2) a.vout2[off] = v;
        }
        // Givens: RHS g of the group on CTA g mod gridDim.x, in the vectors' precision
        for (int g = blockIdx.x; g < gn; g += gridDim.x) {
            if (!gact[g]) continue;                  // uniform over the CTA
            const int r = g0 + g;
            const double hn = sqrt(gn2[g]);
            using C2 = VT;
            C2* col = reinterpret_cast<C2*>(gv);
            C2* csv = col + (J + 2);
            C2* snv = csv + (J + 2);
            double2* csr = a.cs + (long long)r * a.ldg;
            double2* snr = a.sn + (long long)r * a.ldg;
            double2* gr = a.g + (long long)r * a.ldg;
            const double2* h1g = h1 + (size_t)g * nvec;
            for (int k = threadIdx.x; k <= J + 1; k += CT) {
                if (k <= J) a.hsum[(long long)r * a.ldh + k] = h1g[k];
                const double2 hk = k <= J ? h1g[k] : make_double2(hn, 0.0);
                col[k] = mk((Re)hk.x, (Re)hk.y);
                if (k < J) {
                    const double2 ck = HLD(csr + k), sk = HLD(snr + k);
                    csv[k] = mk((Re)ck.x, (Re)0);
                    snv[k] = mk((Re)sk.x, (Re)sk.y);
                }
            }
            __shared__ C2 gpair[2];
            if (threadIdx.x == 0) gpair[0] = mk((Re)HLD(gr + J).x, (Re)HLD(gr + J).y);
            __syncthreads();
            if (threadIdx.x == 0) {
                a.hnorm[r] = hn;
                a.need[r] = gsec[g] ? 1 : 0;
                C2 gj = gpair[0], gj1;
                givens_column<C2>(col, csv, snv, J, gj, gj1);
                gpair[0] = gj;
                gpair[1] = gj1;
                a.invh[r] = hn > 0.0 ? 1.0 / hn : 0.0;
            }
            __syncthreads();
            double2* colg = a.H + r * a.hs + (long long)J * a.ldH;
            for (int k = threadIdx.x; k <= J + 1; k += CT) HST(colg + k, make_double2((double)col[k].x, (double)col[k].y));
            if (threadIdx.x == 32) {
                HST(csr + J, make_double2((double)csv[J].x, 0.0));
                HST(snr + J, make_double2((double)snv[J].x, (double)snv[J].y));
            }
            if (threadIdx.x == 64) {
                const C2 q0 = gpair[0], q1 = gpair[1];
                gr[J] = make_double2((double)q0.x, (double)q0.y);
                gr[J + 1] = make_double2((double)q1.x, (double)q1.y);
                a.est[r] = sqrt((double)q1.x * (double)q1.x + (double)q1.y * (double)q1.y);
            }
            __syncthreads();
        }
        __syncthreads();                             // ws, hv, hc, h1 and the flags are reused by the next group
    }
}

}  // namespace

// Grid size (CTAs, all co-resident) for the persistent Gram-Schmidt kernel, or 0.
int mgs_grid() {
    int dev = 0, sms = 0, per = 0;
    if (cudaGetDevice(&dev) != cudaSuccess) return 0;
    if (cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev) != cudaSuccess) return 0;
    if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per, mgs_kernel<32>, MT, 0) != cudaSuccess) return 0;
    return per >= 1 ? sms : 0;
}

// largest vector length the register-resident kernel handles with `grid` CTAs
long long mgs_max_n(int grid) { return (long long)grid * MT * 32; }

// w <- (w - V V^H w) / ||.|| by modified Gram-Schmidt for every active RHS.
cudaError_t launch_mgs(const double2* V, long long vsk, long long vsr, double2* w, int nvec, long long n, int nrhs,
                       const int* active, double2* hcol, int ldh, double* hnorm, double2* partial, unsigned* bar,
                       int* err, int grid, cudaStream_t st, long long limit) {
    MgsArgs a{V, vsk, vsr, w, nvec, n, nrhs, active, hcol, ldh, hnorm, partial, bar, err,
              limit > 0 ? limit : BAR_LIMIT};
    {
        // basis streamed through shared memory when two slices of every CTA fit; the
        // slice start must stay 16-byte aligned (double2 elements: always)
        const long long L = (n + grid - 1) / grid;
        const long long smem = 2 * L * (long long)sizeof(double2);
        const bool aligned = ((reinterpret_cast<uintptr_t>(V) | reinterpret_cast<uintptr_t>(w)) & 15) == 0 &&
                             ((vsk | vsr) * (long long)sizeof(double2)) % 16 == 0;
        if (aligned && smem <= 220 * 1024 && grid * L >= n) {
            // 256 threads (512 measured 7% slower on the 1023^2 workload: the grid barrier
            // and the reduction cost more than the extra warps hide)
            const long long per = (L + MT - 1) / MT;
            if (per <= 8) return launch_smem_ept<8, MT>(a, grid, (int)L, st);
            if (per <= 16) return launch_smem_ept<16, MT>(a, grid, (int)L, st);
            if (per <= 28) return launch_smem_ept<28, MT>(a, grid, (int)L, st);
        }
    }
    const long long per = (n + (long long)grid * MT - 1) / ((long long)grid * MT);
    if (per <= 4) return launch_ept<4>(a, grid, st);
    if (per <= 8) return launch_ept<8>(a, grid, st);
    if (per <= 16) return launch_ept<16>(a, grid, st);
    if (per <= 32) return launch_ept<32>(a, grid, st);
    return cudaErrorInvalidValue;
}

// shared memory of the fused CGS2 step for a slice of L elements and column j
template <typename VT>
static size_t cgs2_smem(long long L, int j) {
    return (size_t)((j + 2) + (j + 1) + 3 * (j + 2)) * sizeof(double2) + (size_t)((j + 1) + L) * sizeof(VT);
}

// CTAs of the fused CGS2 step for vectors of n elements (~128 elements per CTA, at
// most one CTA per SM), or 0 when a slice does not fit in shared memory
template <typename VT>
int cgs2_grid(long long n, int max_j) {
    const int g = mgs_grid();
    if (g <= 0) return 0;
    // at least 256 elements per CTA: on the 28,644-long interface vectors of the 1023^2,
    // 8 x 8 workload 112 CTAs instead of 152 take 4.62 instead of 4.85 ms of Gram-Schmidt
    // per solve (fewer arrivals per grid barrier); 512 and 1024 measured slower
    const int grid = (int)std::min<long long>(g, std::max<long long>(1, (n + 255) / 256));
    const long long L = (n + grid - 1) / grid;
    return cgs2_smem<VT>(L, max_j) <= 100 * 1024 ? grid : 0;
}

// Column j of the Arnoldi process for every active RHS: CGS2-orthogonalise
// v_{j+1} (in place in V) against v_0..v_j, normalise it, store h_{0..j+1,j}
// and apply the Givens rotations (H, cs, sn, g, est, invh as the Hessenberg step
// kernel leaves them).  partial holds 2 * grid * (j + 2) values.  With dj, j is
// read on the device (*dj, at most jmax) and shared memory is sized for jmax.
// With wsrc, w = -wsrc (the interface operator's output, S v - v); with vout1/2,
// v_{j+1} is also written there (the next step's preconditioner input).  Two or more
// RHS go through cgs2_group_kernel in groups; partial then holds 2 * grid * G * (j + 2)
// values for groups of G <= CG_MAX.
// Launched through cudaLaunchKernelEx with the cooperative attribute, so it can
// be captured into a graph.
template <typename VT>
cudaError_t launch_cgs2_step(const VT* V, long long vsk, long long vsr, int j, long long n, int nrhs,
                             const int* active, double2* hsum, int ldh, double* hnorm, int* need, double2* H, int ldH,
                             long long hs, double2* cs, double2* sn, double2* g, int ldg, double* est, double* invh,
                             double2* partial, unsigned* bar, int* err, int grid, cudaStream_t st, const int* dj,
                             int jmax, const VT* wsrc, VT* vout1, VT* vout2, long long limit, double eta2) {
    if (grid <= 0) return cudaErrorInvalidValue;
    const int L = (int)((n + grid - 1) / grid);
    Cgs2Args<VT> a{V, vsk, vsr, j, n, nrhs, active, hsum, ldh, hnorm, need, H, ldH, hs, cs, sn, g, ldg, est, invh,
                   partial, bar, err, L, dj, wsrc, vout1, vout2, limit > 0 ? limit : BAR_LIMIT, eta2};
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(grid);
    cfg.blockDim = dim3(CT);
    cfg.stream = st;
    cudaLaunchAttribute attr[1];
    attr[0].id = cudaLaunchAttributeCooperative;
    attr[0].val.cooperative = 1;
    cfg.attrs = attr;
    cfg.numAttrs = 1;
    const int J = dj ? jmax : j;
    if (nrhs >= 2) {
        // groups of RHS: as many as fit in ~200 KB of shared memory, at most CG_MAX
        const size_t fixed = (size_t)3 * (J + 2) * sizeof(double2);
        const size_t per = (size_t)((J + 2) + (J + 1)) * sizeof(double2) + (size_t)((J + 1) + L) * sizeof(VT);
        const int G = (int)std::min<long long>(std::min(CG_MAX, nrhs), (long long)((200 * 1024 - fixed) / per));
        if (G >= 2) {
            const size_t smem = fixed + (size_t)G * per;
            cudaError_t e =
                cudaFuncSetAttribute(cgs2_group_kernel<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
            if (e != cudaSuccess) return e;
            cfg.dynamicSmemBytes = smem;
            count_launch();
            return cudaLaunchKernelEx(&cfg, cgs2_group_kernel<VT>, a, G);
        }
    }
    const size_t smem = cgs2_smem<VT>(L, J);
    if (smem > 48 * 1024) {
        cudaError_t e =
            cudaFuncSetAttribute(cgs2_step_kernel<VT>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
        if (e != cudaSuccess) return e;
    }
    cfg.dynamicSmemBytes = smem;
    count_launch();
    return cudaLaunchKernelEx(&cfg, cgs2_step_kernel<VT>, a);
}
#define HELM_CGS2_INST(VT)                                                                                        \
    template int cgs2_grid<VT>(long long, int);                                                                   \
    template cudaError_t launch_cgs2_step<VT>(const VT*, long long, long long, int, long long, int, const int*,   \
                                              double2*, int, double*, int*, double2*, int, long long, double2*,   \
                                              double2*, double2*, int, double*, double*, double2*, unsigned*, int*, \
                                              int, cudaStream_t, const int*, int, const VT*, VT*, VT*, long long, \
                                              double);
HELM_CGS2_INST(double2)
HELM_CGS2_INST(float2)
#undef HELM_CGS2_INST
