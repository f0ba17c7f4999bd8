// Definitions shared by the fused pass kernels (qs_fused.cu: planner and the
// complex64 kernel; qs_fused_ds.cu: the double-single kernel of the
// complex128 state).  See qs_fused.cu for the design of a pass.
#pragma once

#include "qs_internal.cuh"

namespace qs {

constexpr int LB = 5;          // lane bits
#ifndef QS_MAX_WB
#define QS_MAX_WB 3
#endif
constexpr int MAX_WB = QS_MAX_WB;  // warp bits (2^MAX_WB warps per CTA)
constexpr int MAX_OPS = 120;   // ops per pass (shared-memory op table)
#ifndef QS_RB64
#define QS_RB64 5
#endif
#ifndef QS_WB64
#define QS_WB64 3
#endif
#ifndef QS_RB128
#define QS_RB128 4
#endif
#ifndef QS_FUSED_MINBLOCKS
#define QS_FUSED_MINBLOCKS 2
#endif
constexpr int RB64 = QS_RB64;      // complex64: 2^RB64 amplitudes per thread
constexpr int WB64 = QS_WB64;      // complex64: 2^WB64 warps per CTA
constexpr int RB128 = QS_RB128;    // complex128: 2^RB128 amplitudes per thread
// a layout packs RB + WB slots of 4 bits into 32 bits; a control mask over
// the register index is 8 bits wide
static_assert(RB64 + WB64 <= 8 && RB128 + MAX_WB <= 8, "layout does not fit 32 bits");
static_assert(RB64 <= 5 && RB128 <= 5 && MAX_WB <= 4, "register or warp bits out of range");

enum OpType : uint8_t { OP_REG = 0, OP_LANE = 1, OP_DIAG = 2, OP_XPOSE = 3 };

// Fused-only gate class: an uncontrolled Hadamard applied as the butterfly
// (x + y, x - y); the factors 1/sqrt 2 of all such gates of a pass are folded
// into one scale at the store (exact when their number is even, so a complex64
// register does not drift by the rounding of 1/sqrt 2 once per gate).
constexpr int GC_HB = 8;

// One op of the complex64 kernel (112 bytes).
struct alignas(16) POp {
    uint8_t type, cls, tsel, tpos;
    uint8_t rmask, rval;
    uint8_t fast;          // state-vector fast paths: 1 uncontrolled general gate on a register slot,
                           // 2 X deferred into the index mask, 3 uncontrolled general gate on a lane bit
    uint8_t pad0;
    uint32_t pad1;
    uint16_t tmask, tval;
    uint64_t omask, oval;
    // OP_REG / OP_LANE: u00, u01, u10, u11 in c[0..3]; OP_DIAG: d0, d1 in c[0..1]
    //   (the double-single kernel: high parts there, low parts in c[4..7] / c[4..5])
    // OP_XPOSE: 32 uint16 read offsets (old tile order) of the new register
    //           indices in c[0..7], then the old tile-order bit of each new
    //           warp bit (bytes) in c[8..9]
    float2 c[10];
};
static_assert(sizeof(POp) == 112, "POp layout");

struct PassC64 {
    const POp *ops;
    uint64_t tiles;
    int32_t K, WB, nops, has_xpose;
    float scale;                       // folded Hadamard factor (1: none)
    float scale_lo;                    // double-single kernel: low part of the factor
    int32_t n;                         // qubits (trajectory mode: state stride 2^n)
    // trajectory mode: per-(trajectory, op) records; trajectory b's record of
    // op k of this pass is recs[b * rec_stride + rec_off + k]
    const TrajRec *recs;
    uint64_t tiles_per_traj;
    uint32_t rec_stride, rec_off;
    uint8_t tile_pos[24];
    uint64_t ld_reg[32], ld_warp[4];   // global offsets of register index j / warp bit w (first layout)
    uint64_t st_reg[32], st_warp[4];   // the same for the last layout (store)
};

__device__ __forceinline__ bool lpred(int j, uint32_t xm, int rm, int rv) {
    return ((uint32_t(j) ^ xm) & uint32_t(rm)) == uint32_t(rv);
}


// Launches one pass of the double-single kernel (qs_fused_ds.cu) on a
// complex128 state, and the kernel's address for attribute queries.
cudaError_t launch_fused_ds(unsigned grid, unsigned block, size_t smem, cudaStream_t st, double2 *a,
                            const PassC64 &D);
const void *fused_ds_kernel();
constexpr int DS_MINBLOCKS = 1;   // resident CTAs per SM the kernel is built for

}  // namespace qs
