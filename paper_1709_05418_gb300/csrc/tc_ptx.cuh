// tc_ptx.cuh -- inline-PTX wrappers for the sm_100-family tensor-core path used by the
// BF16 network kernel: mbarriers, bulk / tensor (TMA) copies, tensor-memory
// allocation and loads, tcgen05.mma with shared-memory operand descriptors.
#pragma once
#include <cuda_runtime.h>
#include <cstdint>

namespace rpnn {
namespace tc {

// upper bound on polls of one mbarrier phase before a wait gives up (each poll of
// try_wait may itself suspend for a short, hardware-defined time)
constexpr uint32_t kSpinLimit = 1u << 24;
// Suspend-time hint of the issuing thread's polls: a poll whose phase is not complete
// suspends the thread (up to this many ns, or until the phase completes) instead of
// spinning, leaving the scheduler's issue slots to the warps that share it.
constexpr uint32_t kPollHintNs = 256;

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
    return (uint32_t)__cvta_generic_to_shared(p);
}

__device__ __forceinline__ void mbar_init(uint32_t bar, uint32_t count) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], %1;" ::"r"(bar), "r"(count) : "memory");
}
__device__ __forceinline__ void fence_mbar_init() {
    asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
}
__device__ __forceinline__ void mbar_expect_tx(uint32_t bar, uint32_t bytes) {
    asm volatile("mbarrier.arrive.expect_tx.shared::cta.b64 _, [%0], %1;" ::"r"(bar), "r"(bytes) : "memory");
}
__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}
__device__ __forceinline__ bool mbar_test(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n .reg .pred p;\n mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n"
        " selp.u32 %0, 1, 0, p;\n}\n"
        : "=r"(ok) : "r"(bar), "r"(parity) : "memory");
    return ok != 0;
}
// Polls the phase with the given parity at most `limit` times inside one asm statement
// (a C++ loop around a single try_wait costs the issuing thread several hundred cycles
// per wait, which starves the tensor pipe).  Returns the polls left: 0 = not complete.
__device__ __forceinline__ uint32_t mbar_poll(uint32_t bar, uint32_t parity, uint32_t limit) {
    uint32_t left;
    asm volatile(
        "{\n"
        " .reg .pred P1;\n"
        " mov.u32 %0, %3;\n"
        "WAIT_%=:\n"
        " mbarrier.try_wait.parity.shared::cta.b64 P1, [%1], %2, %4;\n"
        " @P1 bra DONE_%=;\n"
        " sub.u32 %0, %0, 1;\n"
        " setp.ne.u32 P1, %0, 0;\n"
        " @P1 bra WAIT_%=;\n"
        "DONE_%=:\n"
        "}\n"
        : "=r"(left) : "r"(bar), "r"(parity), "r"(limit), "r"(kPollHintNs) : "memory");
    return left;
}

// Wait for the phase with the given parity from the thread that issues tcgen05.mma.
// The whole poll loop is one asm statement with no outputs: in that thread, a
// shared-memory load or a wait whose result feeds later code stalls behind the MMAs in
// flight (hundreds of cycles each), and the tensor pipe runs dry.  A poll that fails
// reads the block's abort flag (at shared address abort_addr) and leaves if another role
// has given up; after `limit` failed polls it stores 1 to that flag itself.  Callers
// check the flag later, outside their issue loop.
__device__ __forceinline__ void mbar_wait_issuer(uint32_t bar, uint32_t parity, uint32_t limit,
                                                 uint32_t abort_addr) {
    asm volatile(
        "{\n"
        " .reg .pred P1;\n"
        " .reg .u32 c, f;\n"
        " mov.u32 c, %2;\n"
        "WAIT_%=:\n"
        " mbarrier.try_wait.parity.shared::cta.b64 P1, [%0], %1, %4;\n"
        " @P1 bra DONE_%=;\n"
        " ld.volatile.shared.u32 f, [%3];\n"
        " setp.ne.u32 P1, f, 0;\n"
        " @P1 bra DONE_%=;\n"
        " sub.u32 c, c, 1;\n"
        " setp.ne.u32 P1, c, 0;\n"
        " @P1 bra WAIT_%=;\n"
        " st.volatile.shared.u32 [%3], 1;\n"
        "DONE_%=:\n"
        "}\n" ::"r"(bar), "r"(parity), "r"(limit), "r"(abort_addr), "r"(kPollHintNs) : "memory");
}

// As mbar_wait_issuer, for three barriers at once (each with its own parity): the poll
// succeeds when all three phases have completed.  (Every try_wait costs the issuing thread
// tens of nanoseconds, so a stage waits on exactly the barriers it needs: one, two or three.)
__device__ __forceinline__ void mbar_wait_issuer3(uint32_t b0, uint32_t p0, uint32_t b1, uint32_t p1, uint32_t b2,
                                                  uint32_t p2, uint32_t limit, uint32_t abort_addr) {
    asm volatile(
        "{\n"
        " .reg .pred P1, P2;\n"
        " .reg .u32 c, f;\n"
        " mov.u32 c, %6;\n"
        "WAIT_%=:\n"
        " mbarrier.try_wait.parity.shared::cta.b64 P1, [%0], %1, %8;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 P2, [%2], %3, %8;\n"
        " and.pred P1, P1, P2;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 P2, [%4], %5, %8;\n"
        " and.pred P1, P1, P2;\n"
        " @P1 bra DONE_%=;\n"
        " ld.volatile.shared.u32 f, [%7];\n"
        " setp.ne.u32 P1, f, 0;\n"
        " @P1 bra DONE_%=;\n"
        " sub.u32 c, c, 1;\n"
        " setp.ne.u32 P1, c, 0;\n"
        " @P1 bra WAIT_%=;\n"
        " st.volatile.shared.u32 [%7], 1;\n"
        "DONE_%=:\n"
        "}\n" ::"r"(b0), "r"(p0), "r"(b1), "r"(p1), "r"(b2), "r"(p2), "r"(limit), "r"(abort_addr),
          "r"(kPollHintNs) : "memory");
}

// As mbar_wait_issuer3, for two barriers.
__device__ __forceinline__ void mbar_wait_issuer2(uint32_t b0, uint32_t p0, uint32_t b1, uint32_t p1, uint32_t limit,
                                                  uint32_t abort_addr) {
    asm volatile(
        "{\n"
        " .reg .pred P1, P2;\n"
        " .reg .u32 c, f;\n"
        " mov.u32 c, %4;\n"
        "WAIT_%=:\n"
        " mbarrier.try_wait.parity.shared::cta.b64 P1, [%0], %1, %6;\n"
        " mbarrier.try_wait.parity.shared::cta.b64 P2, [%2], %3, %6;\n"
        " and.pred P1, P1, P2;\n"
        " @P1 bra DONE_%=;\n"
        " ld.volatile.shared.u32 f, [%5];\n"
        " setp.ne.u32 P1, f, 0;\n"
        " @P1 bra DONE_%=;\n"
        " sub.u32 c, c, 1;\n"
        " setp.ne.u32 P1, c, 0;\n"
        " @P1 bra WAIT_%=;\n"
        " st.volatile.shared.u32 [%5], 1;\n"
        "DONE_%=:\n"
        "}\n" ::"r"(b0), "r"(p0), "r"(b1), "r"(p1), "r"(limit), "r"(abort_addr), "r"(kPollHintNs) : "memory");
}

// Bounded wait for the phase with the given parity.  Gives up (returns false) after
// about kSpinLimit polls, or soon after *abort is set by another role of the block.
__device__ __forceinline__ bool mbar_wait(uint32_t bar, uint32_t parity, volatile int* abort) {
    constexpr uint32_t kBurst = 1u << 12;
    for (uint32_t i = 0; i < kSpinLimit / kBurst; ++i) {
        if (mbar_poll(bar, parity, kBurst)) return true;
        if (*abort) return false;
    }
    *abort = 1;
    return false;
}

__device__ __forceinline__ void fence_proxy_async_smem() {
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
}

// 1-D bulk copy global -> shared, completion counted on `bar` (16-byte aligned,
// size a multiple of 16).
__device__ __forceinline__ void bulk_g2s(uint32_t dst, const void* src, uint32_t bytes, uint32_t bar) {
    asm volatile("cp.async.bulk.shared::cluster.global.mbarrier::complete_tx::bytes [%0], [%1], %2, [%3];"
                 ::"r"(dst), "l"(src), "r"(bytes), "r"(bar) : "memory");
}

// 2-D tiled tensor copy global -> shared (box from the tensor map; x in elements of the
// innermost dimension must make x * elem_size a multiple of 16 bytes).
__device__ __forceinline__ void tma_load_2d(uint32_t dst, const void* tmap, int x, int y, uint32_t bar) {
    asm volatile(
        "cp.async.bulk.tensor.2d.shared::cluster.global.tile.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%2, %3}], [%4];"
        ::"r"(dst), "l"(tmap), "r"(x), "r"(y), "r"(bar) : "memory");
}

// ---- tensor memory ---------------------------------------------------------------
__device__ __forceinline__ void tmem_alloc(uint32_t dst_smem, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;"
                 ::"r"(dst_smem), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tmem_relinquish() {
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}

// 32 lanes x 16 consecutive 32-bit columns: thread t of the warp receives lane
// (taddr.lane + t), columns taddr.col .. +15.
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, float v[16]) {
    uint32_t r[16];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 16; ++i) v[i] = __uint_as_float(r[i]);
}

// 32 lanes x 32 consecutive 32-bit columns, waited for inside the same statement so no
// use of the registers can be scheduled before the data has arrived.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, float v[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,"
        "%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%32];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Two 16-column loads, at columns taddr.col and taddr.col + 32, in one round trip:
// v[16 b + i] is column 32 b + i of the thread's lane.
__device__ __forceinline__ void tmem_ld16x2(uint32_t taddr, float v[32]) {
    uint32_t r[32];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%32];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%33];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]),
          "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]),
          "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]),
          "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31])
        : "r"(taddr), "r"(taddr + 32u)
        : "memory");
#pragma unroll
    for (int i = 0; i < 32; ++i) v[i] = __uint_as_float(r[i]);
}

// Seven 16-column loads, at columns taddr.col + 32 b (b = 0..6), in one round trip:
// v[16 b + i] is column 32 b + i of the thread's lane.
__device__ __forceinline__ void tmem_ld16x7(uint32_t taddr, float v[112]) {
    uint32_t r[112];
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%112];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%16,%17,%18,%19,%20,%21,%22,%23,%24,%25,%26,%27,%28,%29,%30,%31}, [%113];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%32,%33,%34,%35,%36,%37,%38,%39,%40,%41,%42,%43,%44,%45,%46,%47}, [%114];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%48,%49,%50,%51,%52,%53,%54,%55,%56,%57,%58,%59,%60,%61,%62,%63}, [%115];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%64,%65,%66,%67,%68,%69,%70,%71,%72,%73,%74,%75,%76,%77,%78,%79}, [%116];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%80,%81,%82,%83,%84,%85,%86,%87,%88,%89,%90,%91,%92,%93,%94,%95}, [%117];\n"
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%96,%97,%98,%99,%100,%101,%102,%103,%104,%105,%106,%107,%108,%109,%110,%111}, [%118];\n"
        "tcgen05.wait::ld.sync.aligned;"
        : "=r"(r[0]), "=r"(r[1]), "=r"(r[2]), "=r"(r[3]), "=r"(r[4]), "=r"(r[5]), "=r"(r[6]), "=r"(r[7]), "=r"(r[8]), "=r"(r[9]), "=r"(r[10]), "=r"(r[11]), "=r"(r[12]), "=r"(r[13]), "=r"(r[14]), "=r"(r[15]), "=r"(r[16]), "=r"(r[17]), "=r"(r[18]), "=r"(r[19]), "=r"(r[20]), "=r"(r[21]), "=r"(r[22]), "=r"(r[23]), "=r"(r[24]), "=r"(r[25]), "=r"(r[26]), "=r"(r[27]), "=r"(r[28]), "=r"(r[29]), "=r"(r[30]), "=r"(r[31]), "=r"(r[32]), "=r"(r[33]), "=r"(r[34]), "=r"(r[35]), "=r"(r[36]), "=r"(r[37]), "=r"(r[38]), "=r"(r[39]), "=r"(r[40]), "=r"(r[41]), "=r"(r[42]), "=r"(r[43]), "=r"(r[44]), "=r"(r[45]), "=r"(r[46]), "=r"(r[47]), "=r"(r[48]), "=r"(r[49]), "=r"(r[50]), "=r"(r[51]), "=r"(r[52]), "=r"(r[53]), "=r"(r[54]), "=r"(r[55]), "=r"(r[56]), "=r"(r[57]), "=r"(r[58]), "=r"(r[59]), "=r"(r[60]), "=r"(r[61]), "=r"(r[62]), "=r"(r[63]), "=r"(r[64]), "=r"(r[65]), "=r"(r[66]), "=r"(r[67]), "=r"(r[68]), "=r"(r[69]), "=r"(r[70]), "=r"(r[71]), "=r"(r[72]), "=r"(r[73]), "=r"(r[74]), "=r"(r[75]), "=r"(r[76]), "=r"(r[77]), "=r"(r[78]), "=r"(r[79]), "=r"(r[80]), "=r"(r[81]), "=r"(r[82]), "=r"(r[83]), "=r"(r[84]), "=r"(r[85]), "=r"(r[86]), "=r"(r[87]), "=r"(r[88]), "=r"(r[89]), "=r"(r[90]), "=r"(r[91]), "=r"(r[92]), "=r"(r[93]), "=r"(r[94]), "=r"(r[95]), "=r"(r[96]), "=r"(r[97]), "=r"(r[98]), "=r"(r[99]), "=r"(r[100]), "=r"(r[101]), "=r"(r[102]), "=r"(r[103]), "=r"(r[104]), "=r"(r[105]), "=r"(r[106]), "=r"(r[107]), "=r"(r[108]), "=r"(r[109]), "=r"(r[110]), "=r"(r[111])
        : "r"(taddr + 0u), "r"(taddr + 32u), "r"(taddr + 64u), "r"(taddr + 96u), "r"(taddr + 128u), "r"(taddr + 160u), "r"(taddr + 192u)
        : "memory");
#pragma unroll
    for (int i = 0; i < 112; ++i) v[i] = __uint_as_float(r[i]);
}

// Store 32 lanes x 16 consecutive 32-bit columns (thread t of the warp writes lane
// taddr.lane + t).  The store is asynchronous: tmem_wait_st() waits for this thread's
// earlier stores to complete.
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const float v[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], {%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15,%16};"
        ::"r"(taddr), "r"(__float_as_uint(v[0])), "r"(__float_as_uint(v[1])), "r"(__float_as_uint(v[2])),
          "r"(__float_as_uint(v[3])), "r"(__float_as_uint(v[4])), "r"(__float_as_uint(v[5])),
          "r"(__float_as_uint(v[6])), "r"(__float_as_uint(v[7])), "r"(__float_as_uint(v[8])),
          "r"(__float_as_uint(v[9])), "r"(__float_as_uint(v[10])), "r"(__float_as_uint(v[11])),
          "r"(__float_as_uint(v[12])), "r"(__float_as_uint(v[13])), "r"(__float_as_uint(v[14])),
          "r"(__float_as_uint(v[15]))
        : "memory");
}
__device__ __forceinline__ void tmem_wait_st() {
    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
}

// ---- descriptors -----------------------------------------------------------------
// Shared-memory matrix descriptor, K-major operand without swizzle: core matrices of 8
// rows x 16 bytes stored as 128 contiguous bytes; `lbo` = byte distance between core
// matrices adjacent along K, `sbo` = byte distance between 8-row groups.
__device__ __forceinline__ uint64_t smem_desc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    uint64_t d = 0;
    d |= (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
    d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
    d |= (uint64_t)1 << 46;               // descriptor version for the sm_100 family
    return d;                              // base offset 0, swizzle none
}

// Shared-memory matrix descriptor, K-major operand with the 64-byte swizzle: rows of 32
// 16-bit elements (64 bytes) at a 64-byte pitch, the 16-byte unit j of row r stored at
// unit j ^ ((r >> 1) & 3); 8-row groups 512 bytes apart; atoms 512-byte aligned.  A
// K-step of 16 elements inside the row is a +32-byte start address.
__device__ __forceinline__ uint64_t smem_desc_sw64(uint32_t addr) {
    uint64_t d = (uint64_t)((addr >> 4) & 0x3FFFu);
    d |= (uint64_t)1 << 16;                // leading offset: unused for swizzled K-major
    d |= (uint64_t)(512u >> 4) << 32;      // 8-row group stride
    d |= (uint64_t)1 << 46;
    d |= (uint64_t)4 << 61;                // 64-byte swizzle
    return d;
}

// Instruction descriptor of kind::f8f6f4: E4M3 A and B (K-major), FP32 accumulator.
__host__ __device__ constexpr uint32_t idesc_e4m3(int M, int N) {
    return (1u << 4)                       // D format: F32
         | (0u << 7)                       // A format: E4M3
         | (0u << 10)                      // B format: E4M3
         | ((uint32_t)(N >> 3) << 17)      // N / 8
         | ((uint32_t)(M >> 4) << 24);     // M / 16
}

// Instruction descriptor of kind::f16: BF16 A and B (K-major), FP32 accumulator.
__host__ __device__ constexpr uint32_t idesc_bf16(int M, int N) {
    return (1u << 4)                       // D format: F32
         | (1u << 7)                       // A format: BF16
         | (1u << 10)                      // B format: BF16
         | ((uint32_t)(N >> 3) << 17)      // N / 8
         | ((uint32_t)(M >> 4) << 24);     // M / 16
}

// D[tmem] (+)= A[smem] * B[smem]^T, one CTA, issued by one thread.
__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t idesc,
                                         uint32_t accumulate) {
    asm volatile(
        "{\n .reg .pred p;\n setp.ne.b32 p, %4, 0;\n"
        " tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n}\n"
        ::"r"(d_tmem), "l"(a), "l"(b), "r"(idesc), "r"(accumulate) : "memory");
}
// Arrive once on `bar` when every previously issued MMA of this thread has completed.
__device__ __forceinline__ void mma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];"
                 ::"r"(bar) : "memory");
}

}  // namespace tc
}  // namespace rpnn
