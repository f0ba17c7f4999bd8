// Fused pass over a complex128 state in double-single arithmetic.
//
// The same pass as the complex64 kernel of qs_fused.cu (tile of 2^13
// amplitudes: 5 lane bits and 8 high bits; 32 amplitudes per thread in
// registers; lane partners by __shfl_xor_sync; transposes through shared
// memory; C-NOTs on register slots deferred into an index mask; every
// layout-dependent offset tabulated on the host), with two differences:
//
//  * the state in memory is complex128; each amplitude is split at the load
//    into two float pairs (re = rh + rl, im = ih + il, 48 significant bits)
//    and joined back into doubles at the store, with integer instructions;
//  * every gate runs in double-single arithmetic (qs_ds.cuh): products of
//    the high parts are exact pairs, sums of them exact pairs, and the
//    low-order terms are added in single precision.  The gate matrices come
//    from the double-precision matrices of the plan, split into high and low
//    floats on the host.
//
// The arithmetic of the pair update (Sec. 2.2.1: x' = u11 x + u12 y,
// y' = u21 x + u22 y) is the same; only the number format differs.  One CTA
// of 256 threads per SM (128 registers of state per thread; a 128 KiB
// transpose buffer).
#include "qs_ds.cuh"
#include "qs_pass.cuh"

namespace qs {

namespace {

using ds::camp;
using ds::ccst;

struct DMat {
    ccst u00, u01, u10, u11;
};

// Matrix of an op: high parts in c[0..3], low parts in c[4..7].
__device__ __forceinline__ DMat load_dmat(const POp &op) {
    const float4 *q = reinterpret_cast<const float4 *>(op.c);
    const float4 h0 = q[0], h1 = q[1], l0 = q[2], l1 = q[3];
    DMat m;
    m.u00 = {h0.x, l0.x, h0.y, l0.y};
    m.u01 = {h0.z, l0.z, h0.w, l0.w};
    m.u10 = {h1.x, l1.x, h1.y, l1.y};
    m.u11 = {h1.z, l1.z, h1.w, l1.w};
    return m;
}

__device__ __forceinline__ camp csel(bool p, const camp &a, const camp &b) {
    return {p ? a.rh : b.rh, p ? a.rl : b.rl, p ? a.ih : b.ih, p ? a.il : b.il};
}

__device__ __forceinline__ camp cshfl(const camp &a, int m) {
    return {__shfl_xor_sync(0xffffffffu, a.rh, m), __shfl_xor_sync(0xffffffffu, a.rl, m),
            __shfl_xor_sync(0xffffffffu, a.ih, m), __shfl_xor_sync(0xffffffffu, a.il, m)};
}

__device__ __forceinline__ bool is_one(const ccst &d) { return d.rh == 1.f && d.rl == 0.f && d.ih == 0.f && d.il == 0.f; }

// General 2x2 on register slot T (matrix roles swapped where the slot is
// deferred-exchanged); with PRED only the pairs whose register bits meet the
// control condition change.
template <int T, bool PRED, int NA>
__device__ __forceinline__ void d_gen(camp (&v)[NA], DMat m, uint32_t xm, int rm, int rv) {
    if ((xm >> T) & 1) {
        ccst t = m.u00; m.u00 = m.u11; m.u11 = t;
        t = m.u01; m.u01 = m.u10; m.u10 = t;
    }
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if ((j >> T) & 1) continue;
        const int j1 = j | (1 << T);
        const camp x = v[j], y = v[j1];
        const camp nx = ds::cmad2(m.u00, x, m.u01, y), ny = ds::cmad2(m.u10, x, m.u11, y);
        if (PRED) {
            const bool p = lpred(j, xm, rm, rv);
            v[j] = csel(p, nx, x);
            v[j1] = csel(p, ny, y);
        } else {
            v[j] = nx;
            v[j1] = ny;
        }
    }
}

template <int T, int NA>
__device__ __forceinline__ void d_xdata(camp (&v)[NA], uint32_t xm, int rm, int rv, bool ok) {
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if ((j >> T) & 1) continue;
        const int j1 = j | (1 << T);
        const bool p = ok && lpred(j, xm, rm, rv);
        const camp x = v[j], y = v[j1];
        v[j] = csel(p, y, x);
        v[j1] = csel(p, x, y);
    }
}

template <int T, int NA>
__device__ __forceinline__ void d_hb(camp (&v)[NA], uint32_t xm) {
    const bool sw = (xm >> T) & 1;
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        if ((j >> T) & 1) continue;
        const int j1 = j | (1 << T);
        camp x = v[j], y = v[j1];
        ds::butterfly(x, y);   // x = sum, y = difference
        const camp nd = {-y.rh, -y.rl, -y.ih, -y.il};
        v[j] = sw ? nd : x;
        v[j1] = sw ? x : y;
    }
}

template <int T, int NA>
__device__ __forceinline__ void d_diag(camp (&v)[NA], const ccst &d0, const ccst &d1, uint32_t xm, int rm, int rv) {
    const bool id0 = is_one(d0), id1 = is_one(d1);
#pragma unroll
    for (int j = 0; j < NA; ++j) {
        const uint32_t l = uint32_t(j) ^ xm;
        const bool hi = (l >> T) & 1;
        if ((hi ? id1 : id0) || (l & uint32_t(rm)) != uint32_t(rv)) continue;
        v[j] = ds::cmul(hi ? d1 : d0, v[j]);
    }
}

template <int T, int NA>
__device__ __forceinline__ void d_reg_op(camp (&v)[NA], int cls, uint32_t &xm, bool ok, int rm, int rv, bool lanectl,
                                         const POp &op) {
    if (cls == GC_X) {
        if (rm == 0 && !lanectl) { xm ^= ok ? (1u << T) : 0u; return; }
        d_xdata<T, NA>(v, xm, rm, rv, ok);
        return;
    }
    if (!ok) return;
    if (cls == GC_HB) { d_hb<T, NA>(v, xm); return; }
    const DMat m = load_dmat(op);
    if (rm) d_gen<T, true, NA>(v, m, xm, rm, rv);
    else d_gen<T, false, NA>(v, m, xm, rm, rv);
}

constexpr int RB = RB64;
constexpr int NA = 1 << RB;

__global__ void __launch_bounds__(32 << WB64, DS_MINBLOCKS) k_fused_ds(double2 *__restrict__ a,
                                                                    const __grid_constant__ PassC64 P) {
    extern __shared__ __align__(16) unsigned char smraw[];
    const int K = P.K, WB = P.WB, nops = P.nops;
    float4 *sm = reinterpret_cast<float4 *>(smraw);
    POp *sops = reinterpret_cast<POp *>(smraw + (P.has_xpose ? (size_t(16) << K) : 0));
    {
        const uint4 *src = reinterpret_cast<const uint4 *>(P.ops);
        uint4 *dst = reinterpret_cast<uint4 *>(sops);
        const int words = nops * int(sizeof(POp) / 16);
        for (int k = threadIdx.x; k < words; k += blockDim.x) dst[k] = src[k];
        __syncthreads();
    }
    const uint32_t tl = threadIdx.x;
    const uint32_t lane = tl & 31u, warp = tl >> 5;
    const int stride = 32 << WB;
    uint64_t ld_t = lane, st_t = lane;
#pragma unroll
    for (int w = 0; w < WB64; ++w)
        if ((warp >> w) & 1) { ld_t += P.ld_warp[w]; st_t += P.st_warp[w]; }

    for (uint64_t tile = blockIdx.x; tile < P.tiles; tile += gridDim.x) {
        uint64_t base = tile;
        for (int k = 0; k < K; ++k) {
            const uint64_t low = (uint64_t(1) << P.tile_pos[k]) - 1;
            base = ((base & ~low) << 1) | (base & low);
        }
        uint32_t xm = 0;
        camp v[NA];
        {
            const double2 *src = a + (base | ld_t);
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                const double2 d = src[P.ld_reg[j]];
                v[j] = ds::load(d.x, d.y);
            }
        }
        for (int k = 0; k < nops; ++k) {
            const POp &op = sops[k];
            const uint4 *q = reinterpret_cast<const uint4 *>(&op);
            const uint4 hd = q[0];
            const int fast = int((hd.y >> 16) & 0xff);
            if (fast) {
                const int tp = hd.x >> 24;
                if (fast == 2) {
                    const uint4 oc = q[1];
                    const uint64_t omask = uint64_t(oc.x) | (uint64_t(oc.y) << 32);
                    const uint64_t oval = uint64_t(oc.z) | (uint64_t(oc.w) << 32);
                    const bool ok = ((tl & (hd.w & 0xffff)) == (hd.w >> 16)) && ((base & omask) == oval);
                    xm ^= ok ? (1u << tp) : 0u;
                    continue;
                }
                const DMat m = load_dmat(op);
                if (fast == 1) {
                    if (tp == 0) d_gen<0, false, NA>(v, m, xm, 0, 0);
                    else if (tp == 1) d_gen<1, false, NA>(v, m, xm, 0, 0);
                    else if (tp == 2) d_gen<2, false, NA>(v, m, xm, 0, 0);
                    else if (tp == 3) d_gen<3, false, NA>(v, m, xm, 0, 0);
                    else d_gen<(RB > 4 ? 4 : 0), false, NA>(v, m, xm, 0, 0);
                } else {
                    const int msk = 1 << tp;
                    const bool hi = (lane >> tp) & 1;
                    const ccst cs = hi ? m.u11 : m.u00, co = hi ? m.u10 : m.u01;
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const camp o = cshfl(v[j], msk);
                        v[j] = ds::cmad2(cs, v[j], co, o);
                    }
                }
                continue;
            }
            const uint4 oc = q[1];
            const int type = hd.x & 0xff, cls = (hd.x >> 8) & 0xff, tsel = (hd.x >> 16) & 0xff,
                      tpos = hd.x >> 24;
            const int rm = hd.y & 0xff, rv = (hd.y >> 8) & 0xff;
            const uint32_t tm = hd.w & 0xffff, tv = hd.w >> 16;
            if (type == OP_XPOSE) {
                const uint32_t cw = (xm * uint32_t(stride)) | tl;
#pragma unroll
                for (int j = 0; j < NA; ++j) {
                    const camp &x = v[j];
                    sm[uint32_t(j * stride) ^ cw] = make_float4(x.rh, x.rl, x.ih, x.il);
                }
                const uint4 *rt = reinterpret_cast<const uint4 *>(op.c);
                uint32_t rd[16];
#pragma unroll
                for (int w4 = 0; w4 < 4; ++w4) {
                    const uint4 t4 = rt[w4];
                    rd[4 * w4] = t4.x; rd[4 * w4 + 1] = t4.y; rd[4 * w4 + 2] = t4.z; rd[4 * w4 + 3] = t4.w;
                }
                const uint4 ow4 = rt[4];
                uint32_t cth = lane;
#pragma unroll
                for (int w = 0; w < WB64; ++w)
                    if (w < WB && ((warp >> w) & 1)) cth |= 1u << ((ow4.x >> (8 * w)) & 0xff);
                __syncthreads();
                xm = 0;
#pragma unroll
                for (int j = 0; j < NA; ++j) {
                    const float4 f = sm[((rd[j >> 1] >> (16 * (j & 1))) & 0xffff) ^ cth];
                    v[j] = {f.x, f.y, f.z, f.w};
                }
                __syncthreads();
                continue;
            }
            const uint64_t omask = uint64_t(oc.x) | (uint64_t(oc.y) << 32);
            const uint64_t oval = uint64_t(oc.z) | (uint64_t(oc.w) << 32);
            const bool ok = ((tl & tm) == tv) && ((base & omask) == oval);
            if (type == OP_REG) {
                const bool lc = (tm & 31u) != 0;
                if (tpos == 0) d_reg_op<0, NA>(v, cls, xm, ok, rm, rv, lc, op);
                else if (tpos == 1) d_reg_op<1, NA>(v, cls, xm, ok, rm, rv, lc, op);
                else if (tpos == 2) d_reg_op<2, NA>(v, cls, xm, ok, rm, rv, lc, op);
                else if (tpos == 3) d_reg_op<3, NA>(v, cls, xm, ok, rm, rv, lc, op);
                else d_reg_op<(RB > 4 ? 4 : 0), NA>(v, cls, xm, ok, rm, rv, lc, op);
            } else if (type == OP_LANE) {
                const int msk = 1 << tpos;
                const bool hi = (lane >> tpos) & 1;
                if (cls == GC_HB) {
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const camp o = cshfl(v[j], msk);
                        // low lane: v + o; high lane: o - v
                        camp s = hi ? o : v[j], t = hi ? v[j] : o;
                        float h, l;
                        ds::add2(s.rh, s.rl, hi ? -t.rh : t.rh, hi ? -t.rl : t.rl, h, l);
                        camp r;
                        r.rh = h; r.rl = l;
                        ds::add2(s.ih, s.il, hi ? -t.ih : t.ih, hi ? -t.il : t.il, h, l);
                        r.ih = h; r.il = l;
                        v[j] = r;
                    }
                } else if (cls == GC_X) {
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const camp o = cshfl(v[j], msk);
                        if (ok && lpred(j, xm, rm, rv)) v[j] = o;
                    }
                } else {
                    const DMat m = load_dmat(op);
                    const ccst cs = hi ? m.u11 : m.u00, co = hi ? m.u10 : m.u01;
#pragma unroll
                    for (int j = 0; j < NA; ++j) {
                        const camp o = cshfl(v[j], msk);
                        if (ok && lpred(j, xm, rm, rv)) v[j] = ds::cmad2(cs, v[j], co, o);
                    }
                }
            } else {  // OP_DIAG
                if (!ok) continue;
                const DMat m = load_dmat(op);
                const ccst d0 = m.u00, d1 = m.u01;
                if (tsel == 0) {
                    if (tpos == 0) d_diag<0, NA>(v, d0, d1, xm, rm, rv);
                    else if (tpos == 1) d_diag<1, NA>(v, d0, d1, xm, rm, rv);
                    else if (tpos == 2) d_diag<2, NA>(v, d0, d1, xm, rm, rv);
                    else if (tpos == 3) d_diag<3, NA>(v, d0, d1, xm, rm, rv);
                    else d_diag<(RB > 4 ? 4 : 0), NA>(v, d0, d1, xm, rm, rv);
                } else {
                    const uint64_t word = tsel == 1 ? uint64_t(tl) : base;
                    const ccst d = ((word >> tpos) & 1) ? d1 : d0;
                    if (is_one(d)) continue;   // this thread's entry is exactly 1
#pragma unroll
                    for (int j = 0; j < NA; ++j)
                        if (lpred(j, xm, rm, rv)) v[j] = ds::cmul(d, v[j]);
                }
            }
        }
        if (P.scale != 1.f || P.scale_lo != 0.f) {
#pragma unroll
            for (int j = 0; j < NA; ++j) {
                camp &x = v[j];
                ds::mul1(x.rh, x.rl, P.scale, P.scale_lo, x.rh, x.rl);
                ds::mul1(x.ih, x.il, P.scale, P.scale_lo, x.ih, x.il);
            }
        }
        double2 *dst = a + (base | st_t);
        uint64_t xg = 0;
#pragma unroll
        for (int r = 0; r < RB; ++r)
            if ((xm >> r) & 1) xg |= P.st_reg[1 << r];
#pragma unroll
        for (int j = 0; j < NA; ++j) {
            const camp &x = v[j];
            dst[P.st_reg[j] ^ xg] = make_double2(ds::join(x.rh, x.rl), ds::join(x.ih, x.il));
        }
    }
}

}  // namespace

cudaError_t launch_fused_ds(unsigned grid, unsigned block, size_t smem, cudaStream_t st, double2 *a,
                            const PassC64 &D) {
    k_fused_ds<<<grid, block, smem, st>>>(a, D);
    return cudaGetLastError();
}

const void *fused_ds_kernel() { return reinterpret_cast<const void *>(&k_fused_ds); }

}  // namespace qs
