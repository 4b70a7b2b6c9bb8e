// Blackwell (sm_103a) building blocks of the tensor-core path: mbarriers,
// TMA tile loads, tcgen05 MMA issue / commit, TMEM allocation and loads, and
// a warp-specialised pipeline shared by every tcgen05 kernel here:
//
//   warp 0, one lane   TMA producer: fills a ring of shared-memory stages
//   warp 1, one lane   MMA issuer:   BF16 x BF16 -> FP32 tcgen05.mma into TMEM
//   warps 2-5          epilogue:     tcgen05.ld of the accumulators (one row
//                                    of the 128-row tile per thread)
//
// Operands are K-major BF16 tiles of 64 elements (128 bytes) per row, loaded
// by TMA with the 128-byte swizzle, which is the canonical K-major SW128
// layout the MMA descriptors below describe (8-row groups 1024 bytes apart).
// Each FP32 operand x is carried as a split pair hi = bf16(x),
// lo = bf16(x - hi); a product uses three MMAs hi*hi + hi*lo + lo*hi into
// one FP32 accumulator (the dropped lo*lo term is below 2^-16 relative).
//
// Every wait is bounded: after about a second it records ST_TIMEOUT in the
// control block, raises the CTA's abort flag and returns false; the roles then
// drain what they have in flight and the CTA releases its TMEM and exits.
#pragma once

#include <cuda.h>
#include <stdint.h>

#include "panda_internal.cuh"

namespace panda {
namespace tc {

constexpr int BM = 128;          // tile rows (TMEM lanes)
constexpr int BK = 64;           // K elements per stage (128 bytes of BF16)
constexpr int THREADS = 192;     // 6 warps
constexpr uint32_t A_BYTES = BM * BK * 2;
constexpr long long WAIT_LIMIT_CYCLES = 2000000000LL;  // ~1 s at 2 GHz

__device__ __forceinline__ uint32_t smem_u32(const void *p)
{
    return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// ---- mbarrier ----------------------------------------------------------------
__device__ __forceinline__ void mbar_init(uint64_t *bar, uint32_t count)
{
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(smem_u32(bar)), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init()
{
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_arrive_expect_tx(uint64_t *bar, uint32_t bytes)
{
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(smem_u32(bar)), "r"(bytes)
                 : "memory");
}
__device__ __forceinline__ bool mbar_try_wait(uint64_t *bar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_u32(bar)), "r"(parity)
        : "memory");
    return ok != 0;
}

// Wait for the phase of `bar` with the given parity.  Gives up after about a
// second (or at once when *abort is set, unless ignore_abort), recording the
// timeout; returns whether the phase completed.
__device__ __forceinline__ bool wait_bounded(uint64_t *bar, uint32_t parity, int *abort, Ctl *ctl,
                                             bool ignore_abort = false)
{
    if (mbar_try_wait(bar, parity))
        return true;
    const long long t0 = clock64();
    while (true) {
        if (mbar_try_wait(bar, parity))
            return true;
        if (!ignore_abort && *(volatile int *)abort)
            return false;
        if (clock64() - t0 > WAIT_LIMIT_CYCLES) {
            atomicExch(abort, 1);
            atomicOr(&ctl->status, ST_TIMEOUT);
            return false;
        }
    }
}

// ---- TMA -------------------------------------------------------------------------
// 2D tile load: inner coordinate x (elements, a multiple of 64 here, so x * 2
// bytes is a multiple of 16), outer coordinate y (rows).
__device__ __forceinline__ void tma_load_2d(void *dst, const CUtensorMap *map, uint64_t *bar, int x, int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"(map), "r"(smem_u32(bar)), "r"(x), "r"(y)
        : "memory");
}

// ---- tcgen05 ----------------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void tc_fence_after() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }

// Shared-memory matrix descriptor of a K-major tile with the 128-byte
// swizzle: start address >> 4 (bits 0-13), leading offset 1 (unused for
// swizzled K-major), stride offset 1024 B >> 4 between 8-row groups (bits
// 32-45), descriptor version 1 (bit 46), layout SWIZZLE_128B = 2 (bits 61-63).
__device__ __forceinline__ uint64_t sdesc_k_sw128(uint32_t saddr)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)1 << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Shared-memory matrix descriptor of an MN-major tile with the 128-byte
// swizzle, as TMA writes a box of 64 MN-contiguous elements by K rows: each K
// row is 128 B (64 BF16 along M or N), 8 rows form a 1024-B swizzle atom.
// Leading offset (bits 16-29) = byte stride between atoms along MN (the next
// 64 elements), stride offset (bits 32-45) = byte stride between 8-row groups
// along K (1024 B); both >> 4.  One MMA of K = 16 spans two K groups, so the
// start address advances by 2048 B per step along K.
__device__ __forceinline__ uint64_t sdesc_mn_sw128(uint32_t saddr, uint32_t mn_atom_bytes)
{
    uint64_t d = 0;
    d |= (uint64_t)((saddr & 0x3FFFFu) >> 4);
    d |= (uint64_t)((mn_atom_bytes >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)(1024 >> 4) << 32;
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)2 << 61;
    return d;
}

// Instruction-descriptor bit that marks the B operand MN-major ("transpose B").
constexpr uint32_t IDESC_B_MN = 1u << 16;
// instruction-descriptor bit for an A operand read MN-major from shared memory
constexpr uint32_t IDESC_A_MN = 1u << 15;

// Instruction descriptor of kind::f16 with BF16 A and B, FP32 accumulator,
// both operands K-major: D format (bits 4-5) = F32, A format (7-9) = BF16,
// B format (10-12) = BF16, N >> 3 (17-22), M >> 4 (24-28).
__host__ __device__ constexpr uint32_t idesc_bf16_f32(int M, int N)
{
    return (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                         uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on `bar` once every tcgen05.mma issued so far by this thread is done.
__device__ __forceinline__ void mma_commit(uint64_t *bar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_u32(bar))
                 : "memory");
}

// 32 consecutive FP32 columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float (&v)[32])
{
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, "
        "%16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]),
          "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]),
          "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 32; ++q)
        v[q] = __uint_as_float(r[q]);
}

// 16 consecutive FP32 columns of this thread's TMEM lane (warp-collective).
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float (&v)[16])
{
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
#pragma unroll
    for (int q = 0; q < 16; ++q)
        v[q] = __uint_as_float(r[q]);
}

// ---- CTA pairs (cta_group::2) ----------------------------------------------------
// Two CTAs of a cluster share one MMA: the even CTA issues it; A (M = 256) is
// split by rows and B (N) by rows between the two CTAs' shared memory, at the
// same offsets; each CTA's TMEM receives its 128 rows of D.
__device__ __forceinline__ uint32_t cluster_ctarank()
{
    uint32_t r;
    asm volatile("mov.u32 %0, %%cluster_ctarank;" : "=r"(r));
    return r;
}
__device__ __forceinline__ void cluster_sync()
{
    asm volatile("barrier.cluster.arrive.release.aligned;\n\tbarrier.cluster.wait.acquire.aligned;" ::: "memory");
}
// shared::cluster address of `addr` (a shared::cta address) in CTA `rank` of the cluster
__device__ __forceinline__ uint32_t mapa_shared(uint32_t addr, uint32_t rank)
{
    uint32_t r;
    asm volatile("mapa.shared::cluster.u32 %0, %1, %2;" : "=r"(r) : "r"(addr), "r"(rank));
    return r;
}
__device__ __forceinline__ void mbar_arrive_cluster(uint32_t cluster_addr)
{
    asm volatile("mbarrier.arrive.release.cluster.shared::cluster.b64 _, [%0];" ::"r"(cluster_addr) : "memory");
}
// TMA load into this CTA's shared memory whose completion is counted on an
// mbarrier of either CTA of the pair (a shared::cluster address).
__device__ __forceinline__ void tma_load_2d_pair(void *dst, const CUtensorMap *map, uint32_t mbar_cluster, int x,
                                                 int y)
{
    asm volatile(
        "cp.async.bulk.tensor.2d.cta_group::2.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1, {%3, %4}], [%2];" ::
            "r"(smem_u32(dst)),
        "l"(map), "r"(mbar_cluster), "r"(x), "r"(y)
        : "memory");
}
__device__ __forceinline__ void tmem_alloc_pair(uint32_t *slot, uint32_t ncols)
{
    asm volatile("tcgen05.alloc.cta_group::2.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_u32(slot)),
                 "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::2.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc_pair(uint32_t taddr, uint32_t ncols)
{
    asm volatile("tcgen05.dealloc.cta_group::2.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void mma_bf16_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
// As mma_bf16_pair, keeping A in the tensor core's collector buffer for the
// next MMA (fill) or reading it from there and releasing it (lastuse): the
// second MMA does not read A from shared memory again.  a_desc is the same.
__device__ __forceinline__ void mma_bf16_pair_fill_a(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                                     uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16.collector::a::fill [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}
__device__ __forceinline__ void mma_bf16_pair_lastuse_a(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc,
                                                        uint32_t idesc, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f16.collector::a::lastuse [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Instruction descriptor of kind::f8f6f4 with E4M3 A and B (format 0 in bits
// 7-9 and 10-12), FP32 accumulator (bits 4-5 = 1), both operands K-major.
__host__ __device__ constexpr uint32_t idesc_e4m3_f32(int M, int N)
{
    return (1u << 4) | ((uint32_t)(N >> 3) << 17) | ((uint32_t)(M >> 4) << 24);
}

// One pair MMA on 8-bit operands: K = 32 per instruction (32 bytes of each
// 128-byte swizzled row, the same byte step as a BF16 MMA's K = 16).
__device__ __forceinline__ void mma_e4m3_pair(uint32_t d_tmem, uint64_t a_desc, uint64_t b_desc, uint32_t idesc,
                                              uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::2.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a_desc), "l"(b_desc), "r"(idesc), "r"(accumulate)
        : "memory");
}

// Arrive on the barrier at this shared offset in both CTAs of the pair once
// the pair's MMAs issued so far are done.
__device__ __forceinline__ void mma_commit_pair(uint64_t *bar)
{
    const uint16_t mask = 0x3;
    asm volatile(
        "tcgen05.commit.cta_group::2.mbarrier::arrive::one.shared::cluster.multicast::cluster.b64 [%0], %1;" ::"r"(
            smem_u32(bar)),
        "h"(mask)
        : "memory");
}

// Start a 16-column TMEM load without waiting (the registers are valid after tmem_wait()).
__device__ __forceinline__ void tmem_ld16_nowait(uint32_t taddr, uint32_t (&r)[16])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]),
          "=r"(r[15])
        : "r"(taddr));
}
__device__ __forceinline__ void tmem_wait() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }
// The wait for a tmem_ld16_nowait into r: r is an in-out operand, so no use of
// it can be scheduled before the loaded values have arrived.
__device__ __forceinline__ void tmem_wait16(uint32_t (&r)[16])
{
    asm volatile("tcgen05.wait::ld.sync.aligned;"
                 : "+r"(r[0]), "+r"(r[1]), "+r"(r[2]), "+r"(r[3]), "+r"(r[4]), "+r"(r[5]), "+r"(r[6]), "+r"(r[7]),
                   "+r"(r[8]), "+r"(r[9]), "+r"(r[10]), "+r"(r[11]), "+r"(r[12]), "+r"(r[13]), "+r"(r[14]),
                   "+r"(r[15])
                 :
                 : "memory");
}

// ---- the pipeline ------------------------------------------------------------------
template <int STAGES>
struct Sync {
    uint64_t full[STAGES];   // TMA -> MMA (transaction bytes)
    uint64_t empty[STAGES];  // MMA -> TMA (tcgen05.commit)
    uint64_t accum;          // MMA -> epilogue (tcgen05.commit after the last k-block)
    uint32_t tmem;           // TMEM base address from tcgen05.alloc
    int abort;               // set on a timed-out wait
    int issued;              // stages the producer issued
    int consumed;            // stages the MMA issuer consumed
};

// Producer: for kb in [0, nk) wait for a free stage and let issue(kb, stage
// base, full barrier) start its four TMA loads.
template <int STAGES, class Issue>
__device__ __forceinline__ void run_producer(Sync<STAGES> &sy, uint8_t *stages, uint32_t stage_bytes, int nk,
                                             Ctl *ctl, Issue issue)
{
    int kb = 0;
    for (; kb < nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
        if (!wait_bounded(&sy.empty[s], ph ^ 1u, &sy.abort, ctl))
            break;
        mbar_arrive_expect_tx(&sy.full[s], stage_bytes);
        issue(kb, stages + (size_t)s * stage_bytes, &sy.full[s]);
    }
    sy.issued = kb;
}

// MMA issuer: for each stage, hi*hi + hi*lo + lo*hi over the 4 K=16 slices
// into the accumulator acc_col(kb) (a TMEM column offset); `first(kb)` says
// whether kb starts a fresh accumulator.  Stage layout: A hi, A lo, B hi, B lo.
template <int STAGES, int BN, class AccCol, class First>
__device__ __forceinline__ void run_mma(Sync<STAGES> &sy, uint8_t *stages, uint32_t stage_bytes, int nk,
                                        Ctl *ctl, AccCol acc_col, First first)
{
    constexpr uint32_t idesc = idesc_bf16_f32(BM, BN);
    constexpr uint32_t B_BYTES = BN * BK * 2;
    int kb = 0;
    for (; kb < nk; ++kb) {
        const int s = kb % STAGES;
        const uint32_t ph = (uint32_t)(kb / STAGES) & 1u;
        if (!wait_bounded(&sy.full[s], ph, &sy.abort, ctl))
            break;
        tc_fence_after();
        const uint32_t base = smem_u32(stages + (size_t)s * stage_bytes);
        const uint32_t d = sy.tmem + acc_col(kb);
        const bool fresh = first(kb);
#pragma unroll
        for (int kk = 0; kk < BK / 16; ++kk) {
            const uint32_t off = kk * 32;  // 16 BF16 = 32 bytes along K inside the swizzled row
            const uint64_t ah = sdesc_k_sw128(base + off);
            const uint64_t al = sdesc_k_sw128(base + A_BYTES + off);
            const uint64_t bh = sdesc_k_sw128(base + 2 * A_BYTES + off);
            const uint64_t bl = sdesc_k_sw128(base + 2 * A_BYTES + B_BYTES + off);
            mma_bf16(d, ah, bh, idesc, (fresh && kk == 0) ? 0u : 1u);
            mma_bf16(d, ah, bl, idesc, 1u);
            mma_bf16(d, al, bh, idesc, 1u);
        }
        mma_commit(&sy.empty[s]);
    }
    sy.consumed = kb;
    mma_commit(&sy.accum);  // also on abort, so the epilogue and the teardown can drain
}

// After the roles are done (all threads past a __syncthreads): make sure no
// TMA load and no MMA is still in flight before the shared memory and TMEM
// are released.  A no-op on the normal path.
template <int STAGES>
__device__ __forceinline__ void drain(Sync<STAGES> &sy, Ctl *ctl)
{
    for (int kb = sy.consumed; kb < sy.issued; ++kb)
        wait_bounded(&sy.full[kb % STAGES], (uint32_t)(kb / STAGES) & 1u, &sy.abort, ctl, true);
}

// Sum v[q] (16 values) over the 32 lanes so that lanes l and l ^ 16 both end
// with the total for q = l & 15 (16 shuffles; fixed order, so deterministic).
__device__ __forceinline__ float lane_transpose_sum16(float (&v)[16])
{
    const int lane = threadIdx.x & 31;
#pragma unroll
    for (int off = 8; off >= 1; off >>= 1) {
        const bool up = (lane & off) != 0;
#pragma unroll
        for (int k = 0; k < off; ++k) {
            const float send = up ? v[k] : v[k + off];
            const float keep = up ? v[k + off] : v[k];
            v[k] = keep + __shfl_xor_sync(0xffffffffu, send, off);
        }
    }
    return v[0] + __shfl_xor_sync(0xffffffffu, v[0], 16);
}

// named barrier among the 256 threads of eight epilogue warps
__device__ __forceinline__ void epi_bar2() { asm volatile("bar.sync 2, 256;" ::: "memory"); }

}  // namespace tc
}  // namespace panda
