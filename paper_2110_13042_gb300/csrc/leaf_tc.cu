// tcgen05 leaf engine: every 128 x 128 output tile of every leaf product
// (diagonal panels, classical tiles, Strassen products) in one persistent
// launch.
//
// Arithmetic (split-digit emulation of a wide product on BF16 tensor cores):
// each operand column is a fixed-point number written as S balanced digits,
//   u = 2^-7 sum_q x_q 2^(-8 (q - 1)),  |x_1| <= 128, x_q in [-128, 127],
// stored in BF16 as x_q 2^(-8 (q - 1)).  The digit products x_p y_q 2^-8(p+q-2)
// are summed on the tensor core into FP32 accumulators in TMEM.  Products
// with the same p + q share one accumulator:
//   acc0: p + q = 2  (1 pair)  |partial| <= 1024 * 2^14      = 2^24 per 1024 rows
//   acc1: p + q = 3  (2 pairs) |partial| <= 2 * 512 * 2^14   = 2^24 per 512 rows
//   acc2: p + q = 4  (3 pairs) |partial| <= 3 * 256 * 2^14   < 2^24 per 256 rows
//   acc3: p + q >= 5 (the rest, weight <= 2^-24 of acc0's unit; not exact)
// so acc0..acc2 hold integers (in their units) below 2^24 and are EXACT in
// FP32 when drained at those intervals.  The epilogue warps drain them into
// a per-element int64 sum T (units of 2^-24 of the leading product), so the
// tile's value is T * 2^(-38 + shift + e_row + e_col) with no rounding
// except the folded low-order digits (acc3) and the final conversion.
//
// Pipeline (one CTA per SM, persistent over a static round-robin task list):
//   warp 0      TMA producer: one 3-D box per operand per stage, all S digit
//               planes of a 128-column x 32-row slab (64-byte swizzle).
//   warp 1      TMEM allocator + single-thread tcgen05.mma issuer.
//   warps 2..9  epilogue: tcgen05.ld drains, int64 accumulation, stores.
// All mbarrier waits are bounded (ptx.cuh).
#include <cuda_bf16.h>
#include <cstdint>

#include "kernels.h"
#include "ptx.cuh"

namespace ata {
namespace {

constexpr int NUM_THREADS = 320;
constexpr int SLICE_BYTES = TILE * KSTEP * 2;  // one digit plane of one operand slab

template <int S>
struct Cfg {
    static constexpr int STAGE_BYTES = 2 * S * SLICE_BYTES;
    static constexpr int STAGES = S == 1 ? 8 : S == 2 ? 6 : S == 3 ? 4 : S == 4 ? 3 : 2;
    static constexpr int NACC = S >= 4 ? 4 : S;
    static constexpr int TMEM_COLS = NACC == 1 ? 128 : NACC == 2 ? 256 : 512;
    static constexpr int BAR_BYTES = 256;
    static constexpr int SMEM_BYTES = 1024 + STAGES * STAGE_BYTES + BAR_BYTES;
    static_assert(SMEM_BYTES <= 232448, "shared memory budget");
};

__host__ __device__ constexpr int acc_of(int p, int q) {
    return (p + q - 2) < 3 ? (p + q - 2) : 3;
}

// Accumulators due for draining at the end of 256-row chunk `c`.
__device__ __forceinline__ uint32_t due_mask(int c, bool last, int nacc) {
    uint32_t m = 1u << 2;                     // acc2 every chunk
    if ((c & 1) == 1 || last) m |= 1u << 1;   // acc1 every 2 chunks
    if ((c & 3) == 3 || last) m |= 1u | (1u << 3);  // acc0, acc3 every 4 chunks
    return m & ((1u << nacc) - 1u);
}

struct Shared {
    uint64_t full[8];
    uint64_t empty[8];
    uint64_t accf;
    uint64_t acce[4];
    uint32_t tmem_base;
    int abort_flag;
};

__device__ __forceinline__ void spin_ns(unsigned long long ns) {
    const unsigned long long t0 = globaltimer_ns();
    while (globaltimer_ns() - t0 < ns) {
    }
}

__device__ __forceinline__ double exp2d(int x) {
    if (x >= -1022 && x <= 1023) return __longlong_as_double(static_cast<long long>(x + 1023) << 52);
    return scalbn(1.0, x);
}
__device__ __forceinline__ float exp2f_(int x) {
    if (x >= -126 && x <= 127) return __uint_as_float(static_cast<unsigned>(x + 127) << 23);
    return scalbnf(1.0f, x);
}

// Add one drained accumulator (32 columns) into T.
template <int ACC>
__device__ __forceinline__ void absorb(int64_t *T, const uint32_t (&r)[32]) {
#pragma unroll
    for (int i = 0; i < 32; ++i) {
        const float v = __uint_as_float(r[i]);
        if (ACC == 0) {
            T[i] += static_cast<int64_t>(__float2int_rn(v)) << 24;
        } else if (ACC == 1) {
            T[i] += static_cast<int64_t>(__float2int_rn(v * 256.0f)) << 16;
        } else if (ACC == 2) {
            T[i] += static_cast<int64_t>(__float2int_rn(v * 65536.0f)) << 8;
        } else {
            T[i] += __float2ll_rn(v * 16777216.0f);
        }
    }
}

template <int S, int ACC>
__device__ __forceinline__ void drain_one(int64_t (&T)[64], uint32_t tbase, int colbase, Shared *sh) {
    uint32_t r[32];
    tmem_ld_32x32b_x32(tbase + ACC * 128 + colbase, r);
    tmem_ld_wait();
    absorb<ACC>(T, r);
    tmem_ld_32x32b_x32(tbase + ACC * 128 + colbase + 32, r);
    tmem_ld_wait();
    tc_fence_before();
    mbar_arrive(&sh->acce[ACC]);
    absorb<ACC>(T + 32, r);
}

template <int S>
__global__ void __maxnreg__(200) leaf_tc_kernel(const __grid_constant__ LeafParams p) {
    using C = Cfg<S>;
    extern __shared__ __align__(1024) uint8_t smem_raw[];
    uint8_t *smem = reinterpret_cast<uint8_t *>((reinterpret_cast<uintptr_t>(smem_raw) + 1023) & ~uintptr_t(1023));
    Shared *sh = reinterpret_cast<Shared *>(smem + C::STAGES * C::STAGE_BYTES);

    const int warp = threadIdx.x >> 5;
    const int lane = threadIdx.x & 31;

    if (threadIdx.x == 0) {
        for (int s = 0; s < C::STAGES; ++s) {
            mbar_init(&sh->full[s], 1);
            mbar_init(&sh->empty[s], 1);
        }
        mbar_init(&sh->accf, 1);
        for (int a = 0; a < 4; ++a) mbar_init(&sh->acce[a], 256);
        sh->abort_flag = 0;
        fence_mbar_init();
    }
    if (warp == 1) {
        tmem_alloc(&sh->tmem_base, C::TMEM_COLS);
        tmem_relinquish();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = sh->tmem_base;
    volatile int *abort_flag = &sh->abort_flag;

    if (warp == 0) {
        // ------------------------------------------------ TMA producer --
        if (lane == 0) {
            int stage = 0;
            uint32_t phase = 0;
            bool ok = true;
            for (int ti = blockIdx.x; ti < p.ntasks && ok; ti += gridDim.x) {
                const LeafTask t = p.tasks[ti];
                const int nsteps = (t.klen + KSTEP - 1) / KSTEP;
                for (int step = 0; step < nsteps; ++step) {
                    if (!mbar_wait(&sh->empty[stage], phase ^ 1u, abort_flag, p.status)) {
                        ok = false;
                        break;
                    }
                    uint8_t *a_dst = smem + stage * C::STAGE_BYTES;
                    uint8_t *b_dst = a_dst + S * SLICE_BYTES;
                    mbar_arrive_expect_tx(&sh->full[stage], C::STAGE_BYTES);
                    const int k = t.k0 + step * KSTEP;
                    tma_load_3d(a_dst, &p.maps[t.fam_u], &sh->full[stage], k, t.col_u, 0);
                    tma_load_3d(b_dst, &p.maps[t.fam_v], &sh->full[stage], k, t.col_v, 0);
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) spin_ns(2000000);  // let copies already in flight land
        }
    } else if (warp == 1) {
        // ------------------------------------------------- MMA issuer --
        if (lane == 0) {
            constexpr uint32_t IDESC = idesc_bf16_f32(TILE, TILE);
            int stage = 0;
            uint32_t phase = 0;
            uint32_t acce_phase = 0;  // bit a: parity of the next acce[a] wait
            uint32_t pending = 0;     // bit a: accumulator a handed to the epilogue
            uint32_t fresh = 0xFu;    // bit a: next MMA into a overwrites
            bool ok = true;
            const uint32_t smem_base = smem_u32(smem);
            for (int ti = blockIdx.x; ti < p.ntasks && ok; ti += gridDim.x) {
                const LeafTask t = p.tasks[ti];
                const int nsteps = (t.klen + KSTEP - 1) / KSTEP;
                for (int step = 0; step < nsteps && ok; ++step) {
                    if (!mbar_wait(&sh->full[stage], phase, abort_flag, p.status)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t a_base = smem_base + stage * C::STAGE_BYTES;
                    const uint32_t b_base = a_base + S * SLICE_BYTES;
                    // Free accumulators first (3, 0, 1, 2); accumulators still
                    // being drained last, in the epilogue's drain order (2, 1, 0, 3).
                    for (int oi = 0; oi < 8 && ok; ++oi) {
                        const int acc = oi < 4 ? ((oi + 3) & 3) : (oi == 4 ? 2 : oi == 5 ? 1 : oi == 6 ? 0 : 3);
                        const bool busy = (pending >> acc) & 1u;
                        if (acc >= C::NACC || busy != (oi >= 4)) continue;
                        if (busy) {
                            if (!mbar_wait(&sh->acce[acc], (acce_phase >> acc) & 1u, abort_flag, p.status)) {
                                ok = false;
                                break;
                            }
                            acce_phase ^= 1u << acc;
                            pending &= ~(1u << acc);
                            tc_fence_after();
                        }
                        const uint32_t d_tmem = tmem + acc * 128;
#pragma unroll
                        for (int pp = 1; pp <= S; ++pp) {
#pragma unroll
                            for (int qq = 1; qq + pp <= S + 1; ++qq) {
                                if (acc_of(pp, qq) != acc) continue;
                                const uint64_t da = sdesc_kmajor_sw64(a_base + (pp - 1) * SLICE_BYTES);
                                const uint64_t db = sdesc_kmajor_sw64(b_base + (qq - 1) * SLICE_BYTES);
#pragma unroll
                                for (int kk = 0; kk < KSTEP / 16; ++kk) {
                                    umma_f16(d_tmem, da + 2 * kk, db + 2 * kk, IDESC,
                                             ((fresh >> acc) & 1u) ? 0u : 1u);
                                    fresh &= ~(1u << acc);
                                }
                            }
                        }
                    }
                    if (!ok) break;
                    umma_commit(&sh->empty[stage]);
                    const bool last = step == nsteps - 1;
                    // Chunk end: hand the due accumulators to the epilogue.  The
                    // most frequently drained accumulator present is due at
                    // every commit and is used by every step, so at most one
                    // accf phase is ever outstanding.
                    const uint32_t due = (last || (step % CHUNK_STEPS) == CHUNK_STEPS - 1)
                                             ? due_mask(step / CHUNK_STEPS, last, C::NACC)
                                             : 0u;
                    if (due) {
                        umma_commit(&sh->accf);
                        pending |= due;
                        fresh |= due;
                    }
                    if (++stage == C::STAGES) {
                        stage = 0;
                        phase ^= 1u;
                    }
                }
            }
            if (!ok) spin_ns(2000000);  // let MMAs already issued retire
        }
    } else {
        // --------------------------------------------------- epilogue --
        const int q = warp & 3;                 // TMEM lane quadrant of this warp
        const int half = (warp - 2) >> 2;       // which 64 columns
        const int row = 32 * q + lane;          // tile row == TMEM lane
        const uint32_t tbase = tmem + (static_cast<uint32_t>(32 * q) << 16);
        const int colbase = 64 * half;
        uint32_t accf_phase = 0;
        bool ok = true;
        for (int ti = blockIdx.x; ti < p.ntasks && ok; ti += gridDim.x) {
            const LeafTask t = p.tasks[ti];
            const int nsteps = (t.klen + KSTEP - 1) / KSTEP;
            const int nchunks = (nsteps + CHUNK_STEPS - 1) / CHUNK_STEPS;
            int64_t T[64];
#pragma unroll
            for (int i = 0; i < 64; ++i) T[i] = 0;
            for (int c = 0; c < nchunks; ++c) {
                const bool last = c == nchunks - 1;
                const uint32_t due = due_mask(c, last, C::NACC);
                if (!due) continue;
                if (!mbar_wait(&sh->accf, accf_phase, abort_flag, p.status)) {
                    ok = false;
                    break;
                }
                accf_phase ^= 1u;
                tc_fence_after();
                if (due & 4u) drain_one<S, 2>(T, tbase, colbase, sh);
                if (due & 2u) drain_one<S, 1>(T, tbase, colbase, sh);
                if (due & 1u) drain_one<S, 0>(T, tbase, colbase, sh);
                if (due & 8u) drain_one<S, 3>(T, tbase, colbase, sh);
            }
            if (!ok) break;
            if (row < t.rows) {
                if (t.kind == OUT_M_I64) {
                    int64_t *out = static_cast<int64_t *>(p.M) + t.out_off + static_cast<int64_t>(row) * t.out_ld;
#pragma unroll
                    for (int i = 0; i < 64; ++i) {
                        const int col = colbase + i;
                        if (col < t.cols) out[col] = T[i];
                    }
                } else {
                    const int er = t.eu >= 0 ? p.expo[t.eu + row] : 0;
                    if (t.kind == OUT_C_F64) {
                        double *out = static_cast<double *>(p.C) + t.out_off + static_cast<int64_t>(row) * t.out_ld;
#pragma unroll
                        for (int i = 0; i < 64; ++i) {
                            const int col = colbase + i;
                            if (col < t.cols && (!t.diag || col <= row)) {
                                const int ec = t.ev >= 0 ? p.expo[t.ev + col] : 0;
                                out[col] = static_cast<double>(T[i]) * exp2d(-38 + t.shift + er + ec);
                            }
                        }
                    } else {
                        float *out = static_cast<float *>(p.C) + t.out_off + static_cast<int64_t>(row) * t.out_ld;
#pragma unroll
                        for (int i = 0; i < 64; ++i) {
                            const int col = colbase + i;
                            if (col < t.cols && (!t.diag || col <= row)) {
                                const int ec = t.ev >= 0 ? p.expo[t.ev + col] : 0;
                                out[col] = __ll2float_rn(T[i]) * exp2f_(-38 + t.shift + er + ec);
                            }
                        }
                    }
                }
            }
        }
    }

    tc_fence_before();
    __syncthreads();
    if (warp == 1) {
        tc_fence_after();
        tmem_dealloc(tmem, C::TMEM_COLS);
    }
}

template <int S>
cudaError_t launch_s(const Plan &P, const LeafParams &lp, int num_sms, cudaStream_t s) {
    using C = Cfg<S>;
    static bool attr_set = false;
    if (!attr_set) {
        cudaError_t e = cudaFuncSetAttribute(leaf_tc_kernel<S>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                             C::SMEM_BYTES);
        if (e != cudaSuccess) return e;
        attr_set = true;
    }
    const int ntasks = static_cast<int>(P.tasks.size());
    const int grid = ntasks < num_sms ? ntasks : num_sms;
    leaf_tc_kernel<S><<<grid, NUM_THREADS, C::SMEM_BYTES, s>>>(lp);
    return cudaGetLastError();
}

}  // namespace

int leaf_tc_smem_bytes(int slices) {
    switch (slices) {
        case 1: return Cfg<1>::SMEM_BYTES;
        case 2: return Cfg<2>::SMEM_BYTES;
        case 3: return Cfg<3>::SMEM_BYTES;
        case 4: return Cfg<4>::SMEM_BYTES;
        case 5: return Cfg<5>::SMEM_BYTES;
        case 6: return Cfg<6>::SMEM_BYTES;
        case 7: return Cfg<7>::SMEM_BYTES;
        default: return 0;
    }
}

cudaError_t launch_leaf_tc(const Plan &P, const LeafParams &lp, int num_sms, cudaStream_t s) {
    if (P.tasks.empty()) return cudaSuccess;
    switch (P.slices) {
        case 1: return launch_s<1>(P, lp, num_sms, s);
        case 2: return launch_s<2>(P, lp, num_sms, s);
        case 3: return launch_s<3>(P, lp, num_sms, s);
        case 4: return launch_s<4>(P, lp, num_sms, s);
        case 5: return launch_s<5>(P, lp, num_sms, s);
        case 6: return launch_s<6>(P, lp, num_sms, s);
        case 7: return launch_s<7>(P, lp, num_sms, s);
        default: return cudaErrorInvalidValue;
    }
}

}  // namespace ata
