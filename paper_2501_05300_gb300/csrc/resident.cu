// Resident projected Jacobi: every sweep of one step in one cooperative kernel.
//
// The sweep of Sec. 2.2 (each contact updated from the previous iterate of its
// two bodies, then every body summing its contacts' impulses) is computed here
// with the arithmetic of the two-pass layout (contact pass + body pass): the
// same contact update, the same shares summed in incidence order.  What
// changes is where the data lives and how the phases are ordered.
//
// One block per SM owns a contiguous range of bodies (slots b0..b1, Morton
// order, so a range is a compact region of the bed), the contacts they own
// and their geometry contacts (contiguous ranges of the contact arrays).  The
// bodies' velocities and the impulse shares of their incidence entries and
// geometry contacts stay in shared memory for all N_it sweeps.  Each sweep has
// a contact phase (every contact and geometry contact of the block, spread
// evenly over the threads, writes its shares) and a body phase (every body sums
// its shares: incidence entries in order, then its geometry contacts, as the
// two-pass body pass adds them).  A contact whose other body lies in another block (a cross contact)
// is computed once, by its owner, which writes that body's share to the global
// share array; a body outside the range is read from the global copy of the
// previous iterate, which its block writes every sweep.
//
// Synchronisation: the contact relation is symmetric, so block X reads data of
// block Y exactly when Y reads data of X: they are neighbours.  Each block
// publishes two counters per sweep (contacts done, bodies done; release store
// after the phase, acquire loads by the neighbours):
//   contact phase of sweep k   after every neighbour's body phase of sweep k-1
//                              (their v^k is written, their reads of the share
//                              slots this phase overwrites are done);
//   body phase of sweep k      after every neighbour's contact phase of sweep k
//                              (the shares of cross contacts are written).
// With two iterate buffers these also order every overwrite of a velocity or
// impulse after the neighbours' last read of the old value.  Every wait is
// bounded: on timeout the block latches DEM_FLAG_TIMEOUT and returns.
#include <algorithm>

#include "dem_internal.cuh"
#include "sweep.cuh"

#define RS_T 1024                  // threads per block
#define RS_SMEM (220 * 1024)       // dynamic shared memory per block [B]
#define RS_MAX_BLOCKS 1024
#define RS_XWORDS (RS_SMEM / 24 / 32 + 1)   // bit mask over the shared share slots

static __device__ __forceinline__ int ld_acquire(const int* p) {
    int v;
    asm volatile("ld.acquire.gpu.global.s32 %0, [%1];" : "=r"(v) : "l"(p) : "memory");
    return v;
}
static __device__ __forceinline__ void st_release(int* p, int v) {
    asm volatile("st.release.gpu.global.s32 [%0], %1;" ::"l"(p), "r"(v) : "memory");
}

// body ranges: block b holds slots floor(b n / G) .. floor((b + 1) n / G) - 1
static __device__ __forceinline__ int range_begin(int b, int n, int G) { return (int)((long long)b * n / G); }
static __device__ __forceinline__ int block_of(int j, int n, int G) {
    return (int)(((long long)(j + 1) * G - 1) / n);
}

// impulse share in shared-memory slot k when `local` and k < icap, else in
// its global slot g (shares of other blocks' bodies are never local)
static __device__ __forceinline__ void put_share(float* sh, bool local, int icap, int k, Imp* g, float3 L, float3 A) {
    if (local && k >= 0 && k < icap) {
        float2* s = reinterpret_cast<float2*>(sh + 6 * (size_t)k);
        s[0] = make_float2(L.x, L.y);
        s[1] = make_float2(L.z, A.x);
        s[2] = make_float2(A.y, A.z);
    } else {
        Imp q;
        q.a = make_float4(L.x, L.y, L.z, A.x);
        q.b = make_float4(A.y, A.z, 0.f, 0.f);
        *g = q;
    }
}

static __device__ __forceinline__ void get_share(const float* sh, bool local, int icap, int k, const Imp* g,
                                                 float3& L, float3& A) {
    if (local && k >= 0 && k < icap) {
        const float2* s = reinterpret_cast<const float2*>(sh + 6 * (size_t)k);
        const float2 a = s[0], b = s[1], c = s[2];
        L = make_float3(a.x, a.y, b.x);
        A = make_float3(b.y, c.x, c.y);
    } else {
        const float4 a = __ldcg(&g->a), b = __ldcg(&g->b);
        L = make_float3(a.x, a.y, a.z);
        A = make_float3(a.w, b.x, b.y);
    }
}

// wait until every neighbour's counter (cnt[q], q in the mask) reaches k;
// false if a wait gave up (or another block latched a fault)
static __device__ bool wait_neighbours(const unsigned* mask, const int* cnt, int G, int k, int* err, int* stop,
                                       unsigned limit) {
    for (int q = threadIdx.x; q < G; q += RS_T) {
        if (!(mask[q >> 5] >> (q & 31) & 1u)) continue;
        unsigned spins = 0;
        while (ld_acquire(&cnt[q]) < k) {
            if (++spins > limit) {
                set_flag(err, DEM_FLAG_TIMEOUT);
                *stop = 1;
                break;
            }
            if ((spins & 255u) == 0u && *(volatile int*)err) {
                *stop = 1;
                break;
            }
            __nanosleep(64);
        }
    }
    __syncthreads();
    return !*stop;
}

static __device__ __forceinline__ void publish(int* cnt, int b, int k) {
    __syncthreads();
    if (threadIdx.x == 0) {
        __threadfence();
        st_release(&cnt[b], k);
    }
}

__global__ void __launch_bounds__(RS_T, 1) k_resident(SimParams P, DevBuf B, ResBuf R, int p, int bcap) {
    extern __shared__ float4 smem[];
    __shared__ unsigned nbmask[RS_MAX_BLOCKS / 32];
    __shared__ int s_stop;
    float4* sv = smem;                                                 // [2 bcap] (v, w) of the bodies
    unsigned* xm = reinterpret_cast<unsigned*>(smem + 2 * bcap);       // [RS_XWORDS] cross-entry bits
    float* sh = reinterpret_cast<float*>(xm + RS_XWORDS);              // [icap] shares, 6 floats each
    const int icap = (int)((RS_SMEM - 32 * (size_t)bcap - 4 * (size_t)RS_XWORDS) / 24);
    const int G = gridDim.x, b = blockIdx.x, n = P.n, tid = threadIdx.x;
    if (*B.err) return;
    const int b0 = range_begin(b, n, G), b1 = range_begin(b + 1, n, G);
    const int nb = b1 - b0;
    const int cbeg = B.own_start[p][b0];
    const int nown = B.own_start[p][b1] - cbeg;
    const int ibase = B.inc_start[b0];
    const int ninc = B.inc_start[b1] - ibase;
    const int gbase = B.geo_start[p][b0];
    const int ngeo = B.geo_start[p][b1] - gbase;
    const int nitem = nown + ngeo;
    const int nit = P.n_it;
    int* cdone = R.prog;        // contact phases finished, per block
    int* bdone = R.prog + G;    // body phases finished, per block

    // prologue: v^0 of the block's bodies, its neighbour blocks, and which
    // entries are cross contacts owned elsewhere (their shares stay global)
    for (int t = tid; t < RS_MAX_BLOCKS / 32; t += RS_T) nbmask[t] = 0u;
    for (int t = tid; t < RS_XWORDS; t += RS_T) xm[t] = 0u;
    if (tid == 0) s_stop = 0;
    __syncthreads();
    for (int k = tid; k < nb; k += RS_T) {
        const int i = b0 + k;
        sv[2 * k] = __ldcg(&B.vw[0][i].v);
        sv[2 * k + 1] = __ldcg(&B.vw[0][i].w);
        const int e1 = B.inc_start[i + 1];
        for (int e = B.inc_start[i]; e < e1; ++e) {
            const int2 ent = B.inc[e];
            const int j = ent.y;
            if (j >= b0 && j < b1) continue;
            const int q = block_of(j, n, G);
            atomicOr(&nbmask[q >> 5], 1u << (q & 31));
            const int k = e - ibase;
            if (ent.x < 0 && k < icap) atomicOr(&xm[k >> 5], 1u << (k & 31));
        }
    }
    __syncthreads();

    for (int it = 0; it < nit; ++it) {
        const int src = it & 1, dst = src ^ 1;
        const bool last = it == nit - 1;
        if (it > 0 && !wait_neighbours(nbmask, bdone, G, it, B.err, &s_stop, P.spin_limit)) return;
        const VW* vin = B.vw[src];
        // contact phase: the block's own contacts, then its geometry contacts;
        // the next item's indices are fetched while this one is computed
        int a_n = 0, bb_n = 0, kg_n = 0;
        int2 pos_n = make_int2(0, 0);
        if (tid < nown) {
            a_n = B.c_self[cbeg + tid];
            bb_n = B.c_other[cbeg + tid];
            pos_n = B.c_pos[cbeg + tid];
        } else if (tid < nitem) {
            kg_n = B.g_body[gbase + tid - nown] - b0;
        }
        for (int q = tid; q < nitem; q += RS_T) {
            const int a = a_n, bb = bb_n, kg = kg_n;
            const int2 pos = pos_n;
            const int qn = q + RS_T;
            if (qn < nown) {
                a_n = B.c_self[cbeg + qn];
                bb_n = B.c_other[cbeg + qn];
                pos_n = B.c_pos[cbeg + qn];
            } else if (qn < nitem) {
                kg_n = B.g_body[gbase + qn - nown] - b0;
            }
            if (q >= nown) {
                const int g = gbase + (q - nown);
                const float4* r = B.grec + 6 * (size_t)g;
                const float4 r0 = r[0], r2 = r[2];
                const float3 nn = f3(r0);
                bool done;
                const Upd u = geom_update(P, B, r, g, src, it, f3(sv[2 * kg]), f3(sv[2 * kg + 1]), done);
                if (done) {
                } else if (last) {
                    write_world(B.glamW[p], g, nn, u);
                } else {
                    B.glamA[dst][g] = make_float4(u.pn, u.pt1, u.pt2, u.pr.x);
                    B.glamB[dst][g] = make_float2(u.pr.y, u.pr.z);
                }
                float3 L, A;
                impulse_a(nn, u.t1, u.t2, r2.x, u.pn, u.pt1, u.pt2, u.pr, L, A);
                put_share(sh, true, icap, ninc + (g - gbase), B.gsh + g, L, A);
                continue;
            }
            const int c = cbeg + q;
            const float4 r0 = B.rec[3 * (size_t)c], r1 = B.rec[3 * (size_t)c + 1], r2 = B.rec[3 * (size_t)c + 2];
            const float4 l0 = __ldcg(&B.lamA[src][c]);
            const float2 l1 = __ldcg(&B.lamB[src][c]);
            const bool bin = bb >= b0 && bb < b1;
            const float4 va = sv[2 * (a - b0)], wa = sv[2 * (a - b0) + 1];
            const float4 vb = bin ? sv[2 * (bb - b0)] : __ldcg(&vin[bb].v);
            const float4 wb = bin ? sv[2 * (bb - b0) + 1] : __ldcg(&vin[bb].w);
            const Upd u = contact_update(r0, r1, r2.x, r2.y, r2.z, r2.w, l0, l1, f3(va) - f3(vb), f3(wa), f3(wb),
                                         P.eps_reg);
            const float3 nn = f3(r0);
            if (last) {
                write_world(B.lamW[p], c, nn, u);
            } else {
                B.lamA[dst][c] = make_float4(u.pn, u.pt1, u.pt2, u.pr.x);
                B.lamB[dst][c] = make_float2(u.pr.y, u.pr.z);
            }
            float3 L = make_float3(0.f, 0.f, 0.f), A = L;
            add_impulse(nn, u.t1, u.t2, r2.x, u.pn, u.pt1, u.pt2, u.pr, false, L, A);
            put_share(sh, true, icap, pos.x - ibase, B.imp + pos.x, L, A);
            L = make_float3(0.f, 0.f, 0.f);
            A = L;
            add_impulse(nn, u.t1, u.t2, r2.y, u.pn, u.pt1, u.pt2, u.pr, true, L, A);
            // a cross contact's share for the other block goes to the global array
            put_share(sh, bin, icap, pos.y - ibase, B.imp + pos.y, L, A);
        }
        publish(cdone, b, it + 1);
        if (!wait_neighbours(nbmask, cdone, G, it + 1, B.err, &s_stop, P.spin_limit)) return;
        // the shares other blocks wrote for this block's bodies, into their shared slots
        const int mcap = min(ninc, icap);
#pragma unroll 4
        for (int m = tid; m < mcap; m += RS_T) {
            if (!(xm[m >> 5] >> (m & 31) & 1u)) continue;
            const float4 x = __ldcg(&B.imp[ibase + m].a), y = __ldcg(&B.imp[ibase + m].b);
            put_share(sh, true, icap, m, nullptr, make_float3(x.x, x.y, x.z), make_float3(x.w, y.x, y.y));
        }
        __syncthreads();
        // body phase: shares in incidence order, then the body's geometry contacts
        for (int k = tid; k < nb; k += RS_T) {
            const int i = b0 + k;
            float3 accL = make_float3(0.f, 0.f, 0.f), accA = accL;
            const int e1 = B.inc_start[i + 1];
            for (int e = B.inc_start[i]; e < e1; ++e) {
                float3 L, A;
                get_share(sh, true, icap, e - ibase, B.imp + e, L, A);
                accL = accL + L;
                accA = accA + A;
            }
            const int g1 = B.geo_start[p][i + 1];
            for (int g = B.geo_start[p][i]; g < g1; ++g) {
                float3 L, A;
                get_share(sh, true, icap, ninc + (g - gbase), B.gsh + g, L, A);
                accL = accL + L;
                accA = accA + A;
            }
            const VW s0 = B.vw0[i];
            const float4 v0 = s0.v, w0 = s0.w;
            const float gm = v0.w > 0.0f ? P.dt : 0.0f;
            const float3 vs = make_float3(v0.x + gm * P.gx, v0.y + gm * P.gy, v0.z + gm * P.gz);
            const float3 v = vs + v0.w * accL;
            const float3 w = f3(w0) + w0.w * accA;
            const float4 ov = make_float4(v.x, v.y, v.z, v0.w), ow = make_float4(w.x, w.y, w.z, w0.w);
            sv[2 * k] = ov;
            sv[2 * k + 1] = ow;
            VW o;
            o.v = ov;
            o.w = ow;
            B.vw[dst][i] = o;
        }
        publish(bdone, b, it + 1);
    }
}

static int res_blocks() {
    static int n = 0;
    if (!n) {
        int dev = 0;
        cudaGetDevice(&dev);
        cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
        if (n <= 0 || n > RS_MAX_BLOCKS) n = -1;
        if (n > 0) {
            // one block per SM must be resident at once (cooperative launch)
            cudaFuncSetAttribute(k_resident, cudaFuncAttributeMaxDynamicSharedMemorySize, RS_SMEM);
            int per_sm = 0;
            if (cudaOccupancyMaxActiveBlocksPerMultiprocessor(&per_sm, k_resident, RS_T, RS_SMEM) != cudaSuccess ||
                per_sm < 1)
                n = -1;
            int coop = 0;
            cudaDeviceGetAttribute(&coop, cudaDevAttrCooperativeLaunch, dev);
            if (!coop) n = -1;
        }
        cudaGetLastError();
    }
    return n;
}

static int body_cap(int n, int G) { return (n + G - 1) / G + 1; }

bool resident_ok(const SimParams& P, int* blocks) {
    const int G = res_blocks();
    if (blocks) *blocks = G;
    if (G <= 0 || P.n < 1 || P.n_it < 1) return false;
    if (P.solver != 0 || P.n_groups > 0 || !P.nit_uniform) return false;
    // the bodies take at most half of the block's shared memory
    return 32LL * body_cap(P.n, G) <= RS_SMEM / 2;
}

int launch_resident(const SimParams& P, const DevBuf& B, const ResBuf& R, int parity, cudaStream_t s) {
    cudaMemsetAsync(R.prog, 0, 2 * R.blocks * sizeof(int), s);
    cudaLaunchConfig_t cfg = {};
    cfg.gridDim = dim3(R.blocks);
    cfg.blockDim = dim3(RS_T);
    cfg.dynamicSmemBytes = RS_SMEM;
    cfg.stream = s;
    cudaLaunchAttribute at[1];
    at[0].id = cudaLaunchAttributeCooperative;
    at[0].val.cooperative = 1;
    cfg.attrs = at;
    cfg.numAttrs = 1;
    cudaLaunchKernelEx(&cfg, k_resident, P, B, R, parity, body_cap(P.n, R.blocks));
    return 1;
}
