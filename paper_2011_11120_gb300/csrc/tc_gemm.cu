// Tensor-core (tcgen05) per-frequency products for the FP16/BF16, split-FP16 and E4M3 kernel
// copies: K-hat and K-hat^H of Eq. 3 when many virtual points make each frequency slice a
// dense GEMM (the batched products the paper uses for groups of focusing points).
//
// The complex product is one real GEMM on the interleaved (re, im) storage of G:
//
//   forward  D[r][n'] = sum_K' G^[r][K'] BT[n'][K'],  K' = 2s + c,
//            BT[2n]   = ( Xr_s, -Xi_s )_s   (row of reals along K')
//            BT[2n+1] = ( Xi_s,  Xr_s )_s
//            -> D[r][2n] = Re Y[r][n], D[r][2n+1] = Im Y[r][n].
//            A = G^ read K-major (rows r contiguous along K').
//   adjoint  D[m][n''] = sum_r G^[r][m] BT[n''][r],  m = 2s + c, n'' = 2n + c'',
//            BT[2n] = (Yr_r)_r, BT[2n+1] = (Yi_r)_r (row scale of G folded in),
//            Re X'[s][n] = D[2s][2n] + D[2s+1][2n+1], Im X'[s][n] = D[2s][2n+1] - D[2s+1][2n].
//            A = the SAME G buffer read MN-major (transposed operand); no second copy.
//
// One CTA computes a 128 x BN tile of D for one frequency: warp 0 streams A and B
// tiles with TMA into a ring of 128-byte-swizzled shared-memory stages, warp 1 (one
// thread) issues tcgen05.mma (M=128, N=BN, K=16, FP32 accumulation in TMEM), warps
// 2-9 read the accumulator back with tcgen05.ld and write complex64 results.  B is
// scaled per (frequency, column) by a power of two so FP16 neither overflows nor
// underflows; the epilogue divides it out and applies G's row scale (forward).
// E4M3 products of at most 21 columns run with the operands swapped (tc_f8_kernel below).
// Every wait on an mbarrier is bounded in wall time: on expiry the thread records
// an error code, the producer drains its own copies in flight, TMEM is freed and
// the CTA exits.
#include <cuda.h>
#include <optional>
#include <cudaTypedefs.h>

#include "common.cuh"

namespace mdc {
namespace {

// warp 0: TMA producer, warp 1: MMA issuer, warps 2..9: epilogue (two warps per TMEM lane
// quarter, each taking half of the accumulator columns); for the E4M3 kernel copy warps
// 10..17 widen each stage's A tile to FP16 and warp 18 streams its bytes
constexpr int TC_THREADS = 320;
constexpr int TC_CVT_THREADS = 256;
// (E4M3) the warp that streams the byte tiles of A, after the converter warps
constexpr int TC_BYTE_WARP = (TC_THREADS + TC_CVT_THREADS) / 32;
constexpr uint32_t TC_STG_BYTES = 128 * 64;     // E4M3 A tile: 128 rows x 64 one-byte reals
constexpr int TC_BM = 128;
constexpr int TC_BK = 64;                       // reduction elements per stage (128 bytes)
// Split format: reduction stages per tensor-core accumulation chunk.  Each chunk's partial sum is
// added into float32 registers by the epilogue (round to nearest), so the tensor core's own
// accumulation spans at most TC_KCHUNK * TC_BK products per output.
constexpr int TC_KCHUNK = 4;
// Bound on the two drain waits before a CTA exits (the producer's copies in flight, the MMA issuer's
// last MMAs).  Those always complete, so this limit is not shortened with the pipeline's limit.
constexpr unsigned long long TC_DRAIN_NS = 2000000000ull;

__device__ __forceinline__ uint32_t su32(const void* p) { return (uint32_t)__cvta_generic_to_shared(p); }
__device__ __forceinline__ unsigned long long gtime() {
    unsigned long long t;
    asm volatile("mov.u64 %0, %%globaltimer;" : "=l"(t));
    return t;
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
// One bounded try: true once the phase with the given parity has completed; the thread may be
// suspended for at most about hint_ns nanoseconds (a hint) while it is not.
__device__ __forceinline__ bool mbar_try(uint32_t bar, uint32_t parity, uint32_t hint_ns) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2, %3;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity), "r"(hint_ns)
        : "memory");
    return ok != 0;
}
// Non-blocking test of the phase with the given parity.
__device__ __forceinline__ bool mbar_poll(uint32_t bar, uint32_t parity) {
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.test_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(bar), "r"(parity)
        : "memory");
    return ok != 0;
}
// Wait for the phase with the given parity to complete, for at most about limit_ns nanoseconds:
// a short spin of non-blocking tests first (hand-offs that complete within a few hundred cycles
// cost no suspension), then tries bounded by a suspend hint no longer than the limit (1 ms at
// most), so the clock is checked at least that often.
__device__ bool mbar_wait(uint32_t bar, uint32_t parity, int* err, int code, unsigned long long limit_ns) {
    for (int i = 0; i < 64; ++i)
        if (mbar_poll(bar, parity)) return true;
    const uint32_t hint = (uint32_t)(limit_ns < 1000000ull ? limit_ns : 1000000ull);
    if (mbar_try(bar, parity, hint)) return true;
    const unsigned long long t0 = gtime();
    for (;;) {
        if (mbar_try(bar, parity, hint)) return true;
        if (gtime() - t0 > limit_ns) {
            atomicCAS(err, 0, code);
            return false;
        }
    }
}
__device__ __forceinline__ void tma_load_3d(uint32_t dst, const CUtensorMap* map, uint32_t bar, int c0,
                                            int c1, int c2) {
    asm volatile(
        "cp.async.bulk.tensor.3d.shared::cluster.global.mbarrier::complete_tx::bytes"
        " [%0], [%1, {%3, %4, %5}], [%2];" ::"r"(dst),
        "l"((unsigned long long)map), "r"(bar), "r"(c0), "r"(c1), "r"(c2)
        : "memory");
}
__device__ __forceinline__ void tc_fence_before() {
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tc_fence_after() {
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
}
__device__ __forceinline__ void tmem_alloc(uint32_t slot, uint32_t ncols) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(slot), "r"(ncols)
                 : "memory");
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
}
__device__ __forceinline__ void tmem_dealloc(uint32_t taddr, uint32_t ncols) {
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(taddr), "r"(ncols) : "memory");
}
// D(tmem) (+)= A(smem desc) * B(smem desc), kind::f16, FP32 accumulation.
__device__ __forceinline__ void umma_f16(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// D(tmem) (+)= A(smem desc) * B(smem desc), kind::f8f6f4 (K = 32 per instruction), FP32 accumulation.
__device__ __forceinline__ void umma_f8(uint32_t d, uint64_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f8f6f4 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d),
        "l"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
// D(tmem) (+)= A(tmem) * B(smem desc), kind::f16: A's row m in TMEM lane m, its 16-bit K elements
// packed two per 32-bit column (even element in the low half).
__device__ __forceinline__ void umma_f16_ta(uint32_t d, uint32_t a, uint64_t b, uint32_t idesc, uint32_t acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "setp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], [%1], %2, %3, p;\n\t}\n" ::"r"(d),
        "r"(a), "l"(b), "r"(idesc), "r"(acc)
        : "memory");
}
__device__ __forceinline__ void tmem_st16(uint32_t taddr, const uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.st.sync.aligned.32x32b.x16.b32 [%0], "
        "{%1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15, %16};" ::"r"(taddr),
        "r"(v[0]), "r"(v[1]), "r"(v[2]), "r"(v[3]), "r"(v[4]), "r"(v[5]), "r"(v[6]), "r"(v[7]), "r"(v[8]),
        "r"(v[9]), "r"(v[10]), "r"(v[11]), "r"(v[12]), "r"(v[13]), "r"(v[14]), "r"(v[15])
        : "memory");
}
__device__ __forceinline__ void umma_commit(uint32_t bar) {
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(bar)
                 : "memory");
}
__device__ __forceinline__ void tmem_ld16(uint32_t taddr, uint32_t (&v)[16]) {
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x16.b32 "
        "{%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, %15}, [%16];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]),
          "=r"(v[15])
        : "r"(taddr));
    asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
}
// Shared-memory matrix descriptor, 128-byte swizzle (layout type 2), descriptor version 1.
__device__ __forceinline__ uint64_t sdesc(uint32_t addr, uint32_t lbo, uint32_t sbo) {
    return (uint64_t)((addr >> 4) & 0x3FFFu) | ((uint64_t)((lbo >> 4) & 0x3FFFu) << 16) |
           ((uint64_t)((sbo >> 4) & 0x3FFFu) << 32) | (1ull << 46) | (2ull << 61);
}

struct TcArgs {
    int nf;             // frequencies (output extent of the bounds checks)
    int kstages;        // reduction slices of TC_BK elements
    int nout;           // output rows: nr (forward) or ns (adjoint)
    int nr;             // kernel rows (row-scale stride)
    int ncol;           // complex columns
    const float* inv_sigma; // [nf][ncol] reciprocals of the power-of-two column scales of B
    const float* gscale;// [nf][nr] kernel row scales (forward epilogue)
    float2* out;
    int ldo, voff_o;
    int* err;
    unsigned long long wait_ns; // bound on every mbarrier wait (wall time)
};

// Pipeline depth: as many stages as fit 198 KB (at most 8); the split format carries two copies.
// The E4M3 path (CVT) keeps three rings: stages of B slices (released when the MMAs that read them
// complete), byte tiles of A (NBY slots, released as soon as they are widened, so the loads of the
// kernel bytes run ahead of the MMAs by the whole byte ring), and WBUF widened FP16 tiles.  The
// byte tiles have 128-byte rows, as many bytes per TMA row as the 16-bit tiles (adjoint: one box
// covers both 64-element halves of the 128 output rows), and for narrow B tiles a stage spans
// KSUB = 2 reduction slices (the widened tile is two slices, each laid out as a 16-bit TMA load of
// one slice would be), halving the hand-offs per kernel byte.
// Reduction slices per E4M3 step for a B tile of BN columns: two for narrow tiles (half the
// hand-offs per kernel byte), one otherwise.
constexpr int tc_cvt_ksub(int bn) { return bn <= 64 ? 2 : 1; }

template <int BN, bool SPLIT, bool CVT = false, bool ADJ = false> struct TcStages {
    static constexpr int KSUB = CVT ? tc_cvt_ksub(BN) : 1;
    // TA: the forward E4M3 product with narrow B tiles widens A into tensor memory (four buffers of
    // KSUB * 32 columns beside the accumulators) instead of shared memory, which leaves shared
    // memory to the TMA byte tiles, their widening reads and B
    static constexpr bool TA = CVT && !ADJ && KSUB == 2;
    // (TA) two independent accumulation chains per tile (even and odd 16-element slices), so that
    // consecutive narrow MMAs do not wait for each other's accumulation; the epilogue adds them
    static constexpr int NCH = TA ? 2 : 1;
    static constexpr int WBUF = TA ? 4 : (CVT ? (KSUB == 2 || BN >= 256 ? 2 : 3) : 0);
    static constexpr int WA = TA ? 0 : TC_BM * 128 * KSUB;            // one widened A tile in shared memory
    static constexpr int TCOLS = TA ? 512 : 2 * BN;                     // TMEM columns allocated
    static constexpr int BYT = CVT ? KSUB * (int)TC_STG_BYTES : 0;     // one byte tile of A
    static constexpr int bytes = CVT ? KSUB * BN * 128 : (SPLIT ? 2 : 1) * (TC_BM * 128 + BN * 128);
    static constexpr int fit = (198 * 1024 - WBUF * WA) / bytes;
    static constexpr int v = TA ? (BN <= 32 ? 8 : 6) : (CVT ? (BN <= 64 ? 4 : 3) : (fit > 8 ? 8 : fit));
    static constexpr int byfit = CVT ? (198 * 1024 - WBUF * WA - v * bytes) / BYT : 0;
    static constexpr int NBY = byfit > 16 ? 16 : byfit;
    static_assert(!CVT || NBY >= 2, "byte ring");
};

template <int BN, bool SPLIT, bool CVT = false, bool ADJ = false>
constexpr size_t tc_smem_bytes() {
    // + alignment, barriers and TMEM slot, two 128-float column-scale buffers, and eight
    // 32 x 20-float output staging tiles
    using S = TcStages<BN, SPLIT, CVT, ADJ>;
    return (size_t)S::v * S::bytes + (size_t)S::NBY * S::BYT + (size_t)S::WBUF * S::WA + 1024 + 512 + 1024 +
           8 * 32 * 20 * 4;
}

// Two E4M3 values (low byte first) to a packed pair of FP16 (exact: E4M3 is a subset of FP16).
__device__ __forceinline__ uint32_t e4m3x2_to_h2(uint32_t w) {
    const __half2_raw r = __nv_cvt_fp8x2_to_halfraw2((__nv_fp8x2_storage_t)(w & 0xffffu), __NV_E4M3);
    return (uint32_t)r.x | ((uint32_t)r.y << 16);
}

// AND of a flag over the 256 epilogue threads (named barrier 2): a failed bounded wait in one
// thread makes all of them leave together, so the named barriers below never miss a thread.
__device__ __forceinline__ bool epilogue_all(bool ok) {
    uint32_t r;
    asm volatile(
        "{\n\t.reg .pred p, q;\n\t"
        "setp.ne.u32 p, %1, 0;\n\t"
        "bar.red.and.pred q, 2, 256, p;\n\t"
        "selp.u32 %0, 1, 0, q;\n\t}"
        : "=r"(r)
        : "r"((uint32_t)ok)
        : "memory");
    return r != 0;
}

__device__ __forceinline__ void mbar_arrive(uint32_t bar) {
    asm volatile("mbarrier.arrive.shared::cta.b64 _, [%0];" ::"r"(bar) : "memory");
}

// Persistent CTA (one per SM): tiles t = blockIdx.x, blockIdx.x + gridDim.x, ... with the
// column tile fastest, then the row tile, then the frequency.  The TMA/MMA stage ring runs
// continuously across tiles and the accumulator is double-buffered in TMEM (2 x BN columns),
// so the epilogue of one tile overlaps the main loop of the next.
//
// CVT (E4M3 kernel copy): warp 18 streams each step's A tile as bytes into a byte ring; warps
// 10..17 widen it to FP16 -- into tensor memory for forward products with narrow B tiles (TA: row
// m in TMEM lane m, the MMA reads A from TMEM), else into the next free tile w of a small
// shared-memory ring laid out as a 16-bit TMA load would have put it (128-byte swizzle) -- then
// release the byte slot and arrive on conv[w]; the MMA issuer waits for the stage (B) and conv[w]
// (A), and its commit frees both.  The MMA is the ordinary kind::f16 with FP16 operands.
template <bool ADJ, int BN, bool SPLIT, bool CVT = false>
__global__ void __launch_bounds__(CVT ? TC_THREADS + TC_CVT_THREADS + 32 : TC_THREADS, 1)
    tc_gemm_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB,
                   const __grid_constant__ CUtensorMap tmA2, const __grid_constant__ CUtensorMap tmB2, TcArgs a,
                   uint32_t idesc, const int* active, int n_tiles_n, int n_tiles_m, int n_tiles) {
    static_assert(!(CVT && SPLIT), "E4M3 widening has no split form");
    if (active && *active == 0) return;
    using SC = TcStages<BN, SPLIT, CVT, ADJ>;
    constexpr int STAGES = SC::v;
    constexpr int WBUF = SC::WBUF;
    constexpr int KSUB = SC::KSUB;
    constexpr int NBY = SC::NBY;
    constexpr uint32_t BYT = SC::BYT;
    constexpr uint32_t A_BYTES = TC_BM * 128;
    constexpr uint32_t B_BYTES = BN * 128;
    constexpr uint32_t WA_BYTES = SC::WA;
    // stage layout: A_hi, B_hi, then (split format) A_lo, B_lo; or (CVT) KSUB B slices
    constexpr uint32_t STAGE_BYTES = SC::bytes;
    // KSUB divides the forward kstages; an adjoint tail slice reads rows past nr (zero filled)
    const int ksteps = (a.kstages + KSUB - 1) / KSUB;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - raw);
    const uint32_t bybase = base + STAGES * STAGE_BYTES;         // (CVT) byte tiles of A
    const uint32_t wbase = bybase + NBY * BYT;                   // (CVT) widened A tiles
    uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + STAGES * STAGE_BYTES + NBY * BYT + WBUF * WA_BYTES);
    // full[STAGES], empty[STAGES], acc_full[2], acc_empty[2], tmem slot (two words), the MMA
    // issuer's drain barrier, (CVT) conv[WBUF], wfree[WBUF], bfull[NBY], bempty[NBY], then the
    // epilogue's double-buffered column scales of the current tile (16-byte aligned)
    constexpr int SIG_OFF = 2 * STAGES + 6 + 2 * WBUF + 2 * NBY;
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * STAGES + 4);
    float* sig_s = reinterpret_cast<float*>(bars + SIG_OFF);
    const uint32_t full0 = su32(bars), empty0 = su32(bars + STAGES);
    const uint32_t accf0 = su32(bars + 2 * STAGES), acce0 = su32(bars + 2 * STAGES + 2);
    const uint32_t drain0 = su32(bars + 2 * STAGES + 5);
    const uint32_t conv0 = su32(bars + 2 * STAGES + 6), wfree0 = conv0 + 8 * WBUF;
    const uint32_t bfull0 = wfree0 + 8 * WBUF, bempty0 = bfull0 + 8 * NBY;
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t_first = (int)blockIdx.x;
    const int t_stride = (int)gridDim.x;
    const unsigned long long wl = a.wait_ns;

    constexpr bool TA = SC::TA;
    constexpr int NCH = SC::NCH;
    constexpr uint32_t ACOL = 2 * NCH * BN;                      // (TA) first TMEM column of the A buffers
    if (warp == 0) tmem_alloc(su32(tmem_slot), SC::TCOLS);
    if (threadIdx.x == 32) {
        for (int i = 0; i < STAGES; ++i) {
            mbar_init(full0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(accf0 + 8 * i, 1);
            mbar_init(acce0 + 8 * i, 256);
        }
        mbar_init(drain0, 1);
        for (int i = 0; i < WBUF; ++i) {
            mbar_init(conv0 + 8 * i, TC_CVT_THREADS / 32);
            mbar_init(wfree0 + 8 * i, 1);
        }
        for (int i = 0; i < NBY; ++i) {
            mbar_init(bfull0 + 8 * i, 1);
            mbar_init(bempty0 + 8 * i, TC_CVT_THREADS / 32);
        }
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;
    const int per_freq = n_tiles_n * n_tiles_m;
    // tile t -> frequency k, first row m0, first column n0
    auto coords = [&](int t, int& k, int& m0, int& n0) {
        k = t / per_freq;
        const int rem = t - k * per_freq;
        const int mt = rem / n_tiles_n;
        m0 = mt * TC_BM;
        n0 = (rem - mt * n_tiles_n) * BN;
    };

    if (warp == 0) {
        if (lane == 0) {
            long g = 0;
            bool ok = true;
            for (int tile = t_first; tile < n_tiles && ok; tile += t_stride) {
                int k, m0, n0;
                coords(tile, k, m0, n0);
                for (int kb = 0; kb < ksteps; ++kb, ++g) {
                    const int s = (int)(g % STAGES);
                    const uint32_t round = (uint32_t)(g / STAGES);
                    if (g >= STAGES && !mbar_wait(empty0 + 8 * s, (round - 1) & 1, a.err, 1, wl)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = base + s * STAGE_BYTES;
                    if constexpr (CVT) {
                        // B slices only: the byte tiles of A come from lane 1
                        mbar_expect_tx(full0 + 8 * s, KSUB * B_BYTES);
#pragma unroll
                        for (int h = 0; h < KSUB; ++h) {
                            const uint32_t bt = sa + h * B_BYTES;
                            const int kx = (kb * KSUB + h) * TC_BK;
                            tma_load_3d(bt, &tmB, full0 + 8 * s, kx, n0, k);
                        }
                        continue;
                    }
                    mbar_expect_tx(full0 + 8 * s, STAGE_BYTES);
#pragma unroll
                    for (int h = 0; h < (SPLIT ? 2 : 1); ++h) {
                        const CUtensorMap* ma = h ? &tmA2 : &tmA;
                        const CUtensorMap* mb = h ? &tmB2 : &tmB;
                        const uint32_t ha = sa + h * (A_BYTES + B_BYTES), hb = ha + A_BYTES;
                        if (!ADJ) {
                            tma_load_3d(ha, ma, full0 + 8 * s, kb * TC_BK, m0, k);
                        } else {
                            tma_load_3d(ha, ma, full0 + 8 * s, m0, kb * TC_BK, k);
                            tma_load_3d(ha + A_BYTES / 2, ma, full0 + 8 * s, m0 + 64, kb * TC_BK, k);
                        }
                        tma_load_3d(hb, mb, full0 + 8 * s, kb * TC_BK, n0, k);
                    }
                }
            }
            // drain: every copy this thread issued must have landed before the CTA can exit
            for (long q = g > STAGES ? g - STAGES : 0; q < g; ++q)
                mbar_wait(full0 + 8 * (int)(q % STAGES), (uint32_t)(q / STAGES) & 1, a.err, 2, TC_DRAIN_NS);
        }
    } else if (CVT && warp == TC_BYTE_WARP) {
        // a warp of its own: a blocking wait of this loop never holds up the B producer
        if (lane == 0) {
            // the byte tiles of A: forward one box of 128 rows x KSUB * 64 bytes, adjoint one box of
            // KSUB * 64 rows x 128 bytes, into slot g % NBY once the converters have released it
            constexpr int NB = NBY > 0 ? NBY : 1;      // (the branch is dead without CVT)
            long g = 0;
            bool ok = true;
            for (int tile = t_first; tile < n_tiles && ok; tile += t_stride) {
                int k, m0, n0;
                coords(tile, k, m0, n0);
                for (int kb = 0; kb < ksteps; ++kb, ++g) {
                    const int y = (int)(g % NB);
                    if (g >= NB && !mbar_wait(bempty0 + 8 * y, (uint32_t)(g / NB - 1) & 1, a.err, 10, wl)) {
                        ok = false;
                        break;
                    }
                    const uint32_t st = bybase + y * BYT;
                    mbar_expect_tx(bfull0 + 8 * y, BYT);
                    // the byte map counts 4-byte elements along its inner dimension
                    if (!ADJ) tma_load_3d(st, &tmA, bfull0 + 8 * y, kb * KSUB * TC_BK / 4, m0, k);
                    else tma_load_3d(st, &tmA, bfull0 + 8 * y, m0 / 4, kb * KSUB * TC_BK, k);
                }
            }
            for (long q = g > NB ? g - NB : 0; q < g; ++q)
                mbar_wait(bfull0 + 8 * (int)(q % NB), (uint32_t)(q / NB) & 1, a.err, 11, TC_DRAIN_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            long g = 0;
            long i = 0;                 // accumulation chunks issued (one per tile unless SPLIT)
            bool ok = true;
            const int kc = SPLIT ? TC_KCHUNK : ksteps;
            for (int tile = t_first; tile < n_tiles && ok; tile += t_stride)
              for (int kb0 = 0; kb0 < ksteps && ok; kb0 += kc, ++i) {
                const int buf = (int)(i & 1);
                if (i >= 2 && !mbar_wait(acce0 + 8 * buf, (uint32_t)((i >> 1) - 1) & 1, a.err, 5, wl)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * NCH * BN);
                const int kb1 = kb0 + kc < ksteps ? kb0 + kc : ksteps;
                for (int kb = kb0; kb < kb1; ++kb, ++g) {
                    const int s = (int)(g % STAGES);
                    if (!mbar_wait(full0 + 8 * s, (uint32_t)(g / STAGES) & 1, a.err, 3, wl)) {
                        ok = false;
                        break;
                    }
                    const int w = CVT ? (int)(g % WBUF) : 0;
                    // CVT: the widened A tile of this step
                    if (CVT && !mbar_wait(conv0 + 8 * w, (uint32_t)(g / (CVT ? WBUF : 1)) & 1, a.err, 7, wl)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = CVT ? wbase + w * WA_BYTES : base + s * STAGE_BYTES;
                    const uint32_t sb = CVT ? base + s * STAGE_BYTES : sa + A_BYTES;
                    const uint32_t sa2 = sb + B_BYTES, sb2 = sa2 + A_BYTES;
                    if constexpr (TA) {
                        // A in TMEM: 8 columns per 16 reduction elements, alternating chains
#pragma unroll
                        for (int kq = 0; kq < KSUB * (TC_BK / 16); ++kq) {
                            const int kk = kq % (TC_BK / 16), ks = kq / (TC_BK / 16);
                            const uint64_t bd = sdesc(sb + ks * B_BYTES + kk * 32, 16, 1024);
                            umma_f16_ta(d + (uint32_t)((kq & 1) * BN), tmem + ACOL + (uint32_t)(w * KSUB * 32 + kq * 8),
                                        bd, idesc, ((kb - kb0) | (kq >> 1)) != 0 ? 1u : 0u);
                        }
                        umma_commit(empty0 + 8 * s);
                        umma_commit(wfree0 + 8 * w);                          // the A buffer is free
                    } else {
#pragma unroll
                        for (int kq = 0; kq < KSUB * (TC_BK / 16); ++kq) {
                            // K-major: +32 bytes per 16 elements inside the swizzled row (next 64-element
                            // slice: next A tile and B slice); MN-major: +16 rows
                            const int kk = kq % (TC_BK / 16), ks = kq / (TC_BK / 16);
                            const uint32_t ao = ks * A_BYTES + (ADJ ? kk * 2048 : kk * 32);
                            const uint32_t lbo = ADJ ? A_BYTES / 2 : 16;
                            const uint64_t ad = sdesc(sa + ao, lbo, 1024);
                            const uint64_t bd = sdesc(sb + ks * B_BYTES + kk * 32, 16, 1024);
                            umma_f16(d, ad, bd, idesc, ((kb - kb0) | kq) != 0 ? 1u : 0u);
                            if (SPLIT) {
                                // hi*lo + lo*hi: the dropped lo*lo term is below 2^-22 relative
                                umma_f16(d, ad, sdesc(sb2 + kk * 32, 16, 1024), idesc, 1u);
                                umma_f16(d, sdesc(sa2 + ao, lbo, 1024), bd, idesc, 1u);
                            }
                        }
                        umma_commit(empty0 + 8 * s);
                        if (CVT) umma_commit(wfree0 + 8 * w);                 // the widened tile is free
                    }
                }
                umma_commit(accf0 + 8 * buf);
              }
            // drain: every MMA this thread issued has completed (it reads shared memory and writes
            // TMEM) before the CTA frees TMEM and exits, also when a wait above gave up
            umma_commit(drain0);
            mbar_wait(drain0, 0, a.err, 9, TC_DRAIN_NS);
        }
    } else if (CVT && warp >= TC_THREADS / 32 && warp < TC_BYTE_WARP) {
        // widen each stage's byte tile: item (row R, 8-byte chunk j) -> 16 bytes at row R, chunk
        // j ^ (R % 8) of the 128-byte-swizzled A tile
        const int ct = threadIdx.x - TC_THREADS;
        // byte tile rows of RB bytes (64 forward with KSUB = 1, else 128).  Forward: 8-byte chunk j
        // of row R goes to slice j / 8, row R; adjoint: row R is reduction row R % 64 of slice R / 64,
        // and chunk j goes to output-row half j / 8 (8 KB apart); in both the widened 16-byte chunk
        // lands swizzled at (j % 8) ^ (R % 8).  Each thread takes 16-byte source chunks (two 8-byte
        // chunks j, j + 1 of one row and slice) whose offsets are the same at every step.
        constexpr int RB = (!ADJ && KSUB == 1) ? 64 : 128;
        constexpr int PER = (int)(KSUB * TC_STG_BYTES) / 16 / TC_CVT_THREADS;
        uint32_t soff[PER], doff[PER][2];
#pragma unroll
        for (int u = 0; u < PER; ++u) {
            const int idx = ct + TC_CVT_THREADS * u;
            const int R = idx / (RB / 16), j = 2 * (idx % (RB / 16));
            const int off = ADJ ? (R >> 6) * (int)A_BYTES + (j >> 3) * (int)(A_BYTES / 2) + (R & 63) * 128
                                : (j >> 3) * (int)A_BYTES + R * 128;
            soff[u] = (uint32_t)(R * RB + j * 8);
            doff[u][0] = (uint32_t)(off + (((j & 7) ^ (R & 7)) << 4));
            doff[u][1] = (uint32_t)(off + ((((j + 1) & 7) ^ (R & 7)) << 4));
        }
        // (TA) this thread widens row R of the byte tile (TMEM lane R: warps reach the lane quarter
        // warp % 4), reduction half hh, into the TMEM A buffer of the step
        const int tq = warp & 3, hh = (warp - TC_THREADS / 32) >> 2, R = 32 * tq + lane;
        long g = 0;
        bool ok = true;
        for (int tile = t_first; tile < n_tiles && ok; tile += t_stride)
            for (int kb = 0; kb < ksteps; ++kb, ++g) {
                const int y = (int)(g % (CVT ? NBY : 1));
                const int w = (int)(g % (CVT ? WBUF : 1));
                if (!mbar_wait(bfull0 + 8 * y, (uint32_t)(g / (CVT ? NBY : 1)) & 1, a.err, 6, wl)) {
                    ok = false;
                    break;
                }
                // the MMAs that read this widened tile on its previous use are complete
                if (g >= WBUF && !mbar_wait(wfree0 + 8 * w, (uint32_t)(g / (CVT ? WBUF : 1) - 1) & 1, a.err, 8, wl)) {
                    ok = false;
                    break;
                }
                const unsigned char* stg = gbase + (bybase - base) + (size_t)y * BYT;
                if constexpr (TA) {
                    // the byte tile arrives 128-byte swizzled: logical 16-byte chunk c of row R sits at
                    // chunk c ^ (R % 8), so the lanes' row reads spread over all banks
                    tc_fence_after();
                    const unsigned char* row = stg + R * 128;
#pragma unroll
                    for (int pass = 0; pass < 2; ++pass) {
                        const int c = 4 * hh + 2 * pass;
                        const uint4 c0 = *reinterpret_cast<const uint4*>(row + ((c ^ (R & 7)) << 4));
                        const uint4 c1 = *reinterpret_cast<const uint4*>(row + (((c + 1) ^ (R & 7)) << 4));
                        const uint32_t b[8] = {c0.x, c0.y, c0.z, c0.w, c1.x, c1.y, c1.z, c1.w};
                        uint32_t v[16];
#pragma unroll
                        for (int i = 0; i < 8; ++i) {
                            v[2 * i] = e4m3x2_to_h2(b[i]);
                            v[2 * i + 1] = e4m3x2_to_h2(b[i] >> 16);
                        }
                        tmem_st16(tmem + ((uint32_t)(32 * tq) << 16) + ACOL + (uint32_t)(w * KSUB * 32 + 32 * hh + 16 * pass), v);
                    }
                    asm volatile("tcgen05.wait::st.sync.aligned;" ::: "memory");
                    tc_fence_before();
                    __syncwarp();
                    if (lane == 0) {
                        mbar_arrive(conv0 + 8 * w);
                        mbar_arrive(bempty0 + 8 * y);
                    }
                    continue;
                }
                unsigned char* at = gbase + (wbase - base) + (size_t)w * WA_BYTES;
                uint4 src[PER];
#pragma unroll
                for (int u = 0; u < PER; ++u) src[u] = *reinterpret_cast<const uint4*>(stg + soff[u]);
#pragma unroll
                for (int u = 0; u < PER; ++u) {
                    uint4 h0, h1;
                    h0.x = e4m3x2_to_h2(src[u].x);
                    h0.y = e4m3x2_to_h2(src[u].x >> 16);
                    h0.z = e4m3x2_to_h2(src[u].y);
                    h0.w = e4m3x2_to_h2(src[u].y >> 16);
                    h1.x = e4m3x2_to_h2(src[u].z);
                    h1.y = e4m3x2_to_h2(src[u].z >> 16);
                    h1.z = e4m3x2_to_h2(src[u].w);
                    h1.w = e4m3x2_to_h2(src[u].w >> 16);
                    *reinterpret_cast<uint4*>(at + doff[u][0]) = h0;
                    *reinterpret_cast<uint4*>(at + doff[u][1]) = h1;
                }
                // the tensor core reads the tile through the async proxy
                asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
                __syncwarp();
                if (lane == 0) {
                    mbar_arrive(conv0 + 8 * w);
                    mbar_arrive(bempty0 + 8 * y);      // this warp's reads of the byte tile are done
                }
            }
    } else {
        const int q = warp & 3;                  // TMEM lane quarter of this warp
        const int row = q * 32 + lane;
        constexpr int BH = BN / 2;               // accumulator columns per epilogue warp
        const int cbeg = ((warp - 2) >> 2) * BH;
        long i = 0;                     // accumulation chunks consumed
        const int nch = SPLIT ? (a.kstages + TC_KCHUNK - 1) / TC_KCHUNK : 1;
        int parity = 0;
        for (int tile = t_first; tile < n_tiles; tile += t_stride, parity ^= 1) {
            int k, m0, n0;
            coords(tile, k, m0, n0);
            // this tile's reciprocal column scales (exact: powers of two) into shared memory; the
            // buffer alternates with the tile parity so the next tile's copy never races a reader
            float* sgs = sig_s + parity * 128;
            {
                const int e = threadIdx.x - 64;
                const int n = (n0 >> 1) + e;
                if (e < BN / 2)
                    sgs[e] = n < a.ncol && MDC_INB((size_t)k * a.ncol + n, 1, (long long)a.nf * a.ncol, a.err, 131)
                                 ? a.inv_sigma[(size_t)k * a.ncol + n] : 0.f;
                asm volatile("bar.sync 1, 256;" ::: "memory");
            }
            const int r = m0 + row;
            const float gs = (!ADJ && r < a.nout && MDC_INB((size_t)k * a.nr + r, 1, (long long)a.nf * a.nr, a.err, 132))
                                 ? a.gscale[(size_t)k * a.nr + r] : 1.f;
            // Store 16 accumulator columns c0.. (8 complex output columns) of this warp's 32 rows:
            // scaled values go through a per-warp staging tile (rows padded to 20 floats, so both
            // the row-wise writes and the column-wise reads are conflict-free), then each store
            // instruction writes 8 output rows x 64 contiguous bytes.
            float* stg = sig_s + 256 + (warp - 2) * (32 * 20);
            auto emit = [&](int c0, const float* v) {
                const int nb = (n0 + c0) >> 1;
                float w[16];
                if (!ADJ) {
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float f = gs * sgs[(c0 >> 1) + j];
                        w[2 * j] = v[2 * j] * f;
                        w[2 * j + 1] = v[2 * j + 1] * f;
                    }
                } else {
                    // rows 2s and 2s + 1 of the real product hold the two halves of output row s
                    float pv[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) pv[j] = __shfl_xor_sync(0xffffffffu, v[j], 1);
#pragma unroll
                    for (int j = 0; j < 8; ++j) {
                        const float f = sgs[(c0 >> 1) + j];
                        w[2 * j] = (v[2 * j] + pv[2 * j + 1]) * f;
                        w[2 * j + 1] = (v[2 * j + 1] - pv[2 * j]) * f;
                    }
                }
                constexpr int NROWS = ADJ ? 16 : 32;
                const int orow0 = ADJ ? (m0 + 32 * q) >> 1 : m0 + 32 * q;
                if (!ADJ || (lane & 1) == 0) {
                    float* rowp = stg + (ADJ ? lane >> 1 : lane) * 20;
#pragma unroll
                    for (int i4 = 0; i4 < 4; ++i4)
                        *reinterpret_cast<float4*>(rowp + 4 * i4) =
                            make_float4(w[4 * i4], w[4 * i4 + 1], w[4 * i4 + 2], w[4 * i4 + 3]);
                }
                __syncwarp();
                const int cc = lane >> 3, n = nb + 2 * cc;
#pragma unroll
                for (int it = 0; it < NROWS / 8; ++it) {
                    const int rr = (lane & 7) + 8 * it, orow = orow0 + rr;
                    const float4 val = *reinterpret_cast<const float4*>(stg + rr * 20 + 4 * cc);
                    if (orow < a.nout && n < a.ncol &&
                        MDC_INB(((size_t)k * a.nout + orow) * a.ldo + a.voff_o + n, n + 1 < a.ncol ? 2 : 1,
                                (long long)a.nf * a.nout * a.ldo, a.err, 130)) {
                        float2* dst = a.out + ((size_t)k * a.nout + orow) * a.ldo + a.voff_o + n;
                        if (n + 1 < a.ncol && (reinterpret_cast<uintptr_t>(dst) & 15) == 0) {
                            *reinterpret_cast<float4*>(dst) = val;
                        } else {
                            dst[0] = make_float2(val.x, val.y);
                            if (n + 1 < a.ncol) dst[1] = make_float2(val.z, val.w);
                        }
                    }
                }
                __syncwarp();
            };
            bool ok = true;
            if constexpr (SPLIT) {
                // sum the chunks' partial accumulators in float32 registers, then store
                float acc[BH];
#pragma unroll
                for (int c = 0; c < BH; ++c) acc[c] = 0.f;
                for (int ch = 0; ch < nch; ++ch, ++i) {
                    const int buf = (int)(i & 1);
                    if (!epilogue_all(mbar_wait(accf0 + 8 * buf, (uint32_t)(i >> 1) & 1, a.err, 4, wl))) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * BN);
#pragma unroll
                    for (int c0 = 0; c0 < BH; c0 += 16) {
                        uint32_t v[16];
                        tmem_ld16(taddr + cbeg + c0, v);
#pragma unroll
                        for (int j = 0; j < 16; ++j) acc[c0 + j] += __uint_as_float(v[j]);
                    }
                    tc_fence_before();
                    mbar_arrive(acce0 + 8 * buf);
                }
                if (!ok) break;
#pragma unroll
                for (int c0 = 0; c0 < BH; c0 += 16) emit(cbeg + c0, acc + c0);
            } else {
                const int buf = (int)(i & 1);
                if (!epilogue_all(mbar_wait(accf0 + 8 * buf, (uint32_t)(i >> 1) & 1, a.err, 4, wl))) break;
                tc_fence_after();
                const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * NCH * BN);
#pragma unroll 1
                for (int c0 = cbeg; c0 < cbeg + BH; c0 += 16) {
                    uint32_t v[16];
                    tmem_ld16(taddr + c0, v);
                    float f[16];
#pragma unroll
                    for (int j = 0; j < 16; ++j) f[j] = __uint_as_float(v[j]);
                    if constexpr (NCH == 2) {
                        tmem_ld16(taddr + BN + c0, v);
#pragma unroll
                        for (int j = 0; j < 16; ++j) f[j] += __uint_as_float(v[j]);
                    }
                    emit(c0, f);
                }
                tc_fence_before();
                mbar_arrive(acce0 + 8 * buf);
                ++i;
            }
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, SC::TCOLS);
    }
}

// ------------------------------------------------------------------ E4M3 products, operands swapped
// With few columns the product above issues M = 128 x N = 2 ncol MMAs (N = 32 at 16 columns), and
// their instruction rate, not the kernel's bytes, bounds it.  Here the kernel is the N = 256
// operand, read as E4M3 bytes straight from its copy (kind::f8f6f4, no widening), and the spectra
// are the M operand: each real row of the B operand above is split exactly into three E4M3 terms,
//     sigma x = h0 + h1 / 16 + h2 / 256   (round to nearest even at each step),
// stacked as rows t * R + row (R = 2 ncol, 3R <= 128) of one 128-row tile, so one MMA per 32
// reduction elements forms all three partial products, in different TMEM lanes.  The epilogue adds
// them with their weights (about 12 significant bits of the spectra, finer than the FP16 rounding
// of the 16-bit path) and applies the scales.
//   forward  D'[t R + 2n + c][r]  = sum_K' A[t R + 2n + c][K'] G^[r][K']   (G^ K-major, N = r)
//            rows 2n: (Re, -Im), 2n + 1: (Im, Re) of X column n along s; Y[k][r][n] = D'[2n][r] +
//            i D'[2n + 1][r] (term-weighted), times G's row scale and 1 / sigma.
//   adjoint  D'[t R + 2n + c][m] = sum_r A[t R + 2n + c][r] G^[r][m]      (G^ MN-major, N = m = 2s + c')
//            rows 2n: Re, 2n + 1: Im of Y column n times G's row scale, along r;
//            X'[k][s][n] = (D'[2n][2s] + D'[2n+1][2s+1]) + i (D'[2n+1][2s] - D'[2n][2s+1]), times 1 / sigma.
constexpr int F8_BN = 256;                          // kernel rows per tile (N of the MMA)
constexpr int F8_STAGES = 4;
constexpr uint32_t F8_A_BYTES = TC_BM * 128;        // stacked spectra terms: 128 rows x 128 bytes
constexpr uint32_t F8_B_BYTES = F8_BN * 128;        // kernel bytes: 256 rows x 128 bytes
constexpr uint32_t F8_STAGE = F8_A_BYTES + F8_B_BYTES;
constexpr int F8_TERMS = 3;
constexpr int F8_MAX_COLS = TC_BM / (2 * F8_TERMS);   // 21 columns: 3 terms x 42 rows fit 128
constexpr int F8_LD = 17;                           // epilogue staging row pitch (floats)

constexpr size_t f8_smem_bytes() {
    // + alignment, barriers, and two 128 x 17-float staging tiles (one per column half)
    return (size_t)F8_STAGES * F8_STAGE + 1024 + 256 + 2 * TC_BM * F8_LD * 4;
}

// Persistent CTA (one per SM) over tiles (frequency k, N columns n0 .. n0 + 255: kernel rows forward,
// interleaved kernel columns adjoint): warp 0 streams each 128-element reduction slice of the stacked
// spectra (128 rows x 128 bytes) and of the kernel (forward 256 rows x 128 bytes; adjoint 128 rows
// x 2 x 128 bytes, the two 128-column halves 16 KB apart) with TMA, warp 1 issues four MMAs per
// slice into one of two TMEM accumulators, warps 2..9 read the other back (4 lane quarters x 2
// column halves), add the terms through shared memory and store.  Every wait is bounded as in
// tc_gemm_kernel.
template <bool ADJ>
__global__ void __launch_bounds__(TC_THREADS, 1)
    tc_f8_kernel(const __grid_constant__ CUtensorMap tmA, const __grid_constant__ CUtensorMap tmB, TcArgs a,
                 uint32_t idesc, const int* active, int n_tiles_n, int n_tiles) {
    if (active && *active == 0) return;
    const int ksteps = a.kstages;
    extern __shared__ __align__(1024) unsigned char smem_raw[];
    const uint32_t raw = su32(smem_raw);
    const uint32_t base = (raw + 1023u) & ~1023u;
    unsigned char* gbase = smem_raw + (base - raw);
    // full[S], empty[S], acc_full[2], acc_empty[2], tmem slot, drain; staging tiles 256 bytes on
    uint64_t* bars = reinterpret_cast<uint64_t*>(gbase + F8_STAGES * F8_STAGE);
    uint32_t* tmem_slot = reinterpret_cast<uint32_t*>(bars + 2 * F8_STAGES + 4);
    float* stg = reinterpret_cast<float*>(bars + 32);
    const uint32_t full0 = su32(bars), empty0 = su32(bars + F8_STAGES);
    const uint32_t accf0 = su32(bars + 2 * F8_STAGES), acce0 = su32(bars + 2 * F8_STAGES + 2);
    const uint32_t drain0 = su32(bars + 2 * F8_STAGES + 5);
    const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
    const int t_first = (int)blockIdx.x, t_stride = (int)gridDim.x;
    const unsigned long long wl = a.wait_ns;

    if (warp == 0) tmem_alloc(su32(tmem_slot), 2 * F8_BN);
    if (threadIdx.x == 32) {
        for (int i = 0; i < F8_STAGES; ++i) {
            mbar_init(full0 + 8 * i, 1);
            mbar_init(empty0 + 8 * i, 1);
        }
        for (int i = 0; i < 2; ++i) {
            mbar_init(accf0 + 8 * i, 1);
            mbar_init(acce0 + 8 * i, 256);
        }
        mbar_init(drain0, 1);
        fence_mbar_init();
    }
    tc_fence_before();
    __syncthreads();
    tc_fence_after();
    const uint32_t tmem = *tmem_slot;

    if (warp == 0) {
        if (lane == 0) {
            long g = 0;
            bool ok = true;
            for (int tile = t_first; tile < n_tiles && ok; tile += t_stride) {
                const int k = tile / n_tiles_n, n0 = (tile - k * n_tiles_n) * F8_BN;
                for (int kb = 0; kb < ksteps; ++kb, ++g) {
                    const int s = (int)(g % F8_STAGES);
                    if (g >= F8_STAGES &&
                        !mbar_wait(empty0 + 8 * s, (uint32_t)(g / F8_STAGES - 1) & 1, a.err, 1, wl)) {
                        ok = false;
                        break;
                    }
                    const uint32_t sa = base + s * F8_STAGE;
                    mbar_expect_tx(full0 + 8 * s, F8_STAGE);
                    // the maps count 4-byte elements along their inner (byte) dimension
                    tma_load_3d(sa, &tmA, full0 + 8 * s, kb * 32, 0, k);
                    if (!ADJ) {
                        tma_load_3d(sa + F8_A_BYTES, &tmB, full0 + 8 * s, kb * 32, n0, k);
                    } else {
                        tma_load_3d(sa + F8_A_BYTES, &tmB, full0 + 8 * s, n0 / 4, kb * 128, k);
                        tma_load_3d(sa + F8_A_BYTES + F8_B_BYTES / 2, &tmB, full0 + 8 * s, (n0 + 128) / 4, kb * 128, k);
                    }
                }
            }
            // drain: every copy this thread issued must have landed before the CTA can exit
            for (long q = g > F8_STAGES ? g - F8_STAGES : 0; q < g; ++q)
                mbar_wait(full0 + 8 * (int)(q % F8_STAGES), (uint32_t)(q / F8_STAGES) & 1, a.err, 2, TC_DRAIN_NS);
        }
    } else if (warp == 1) {
        if (lane == 0) {
            long g = 0, i = 0;
            bool ok = true;
            for (int tile = t_first; tile < n_tiles && ok; tile += t_stride, ++i) {
                const int buf = (int)(i & 1);
                if (i >= 2 && !mbar_wait(acce0 + 8 * buf, (uint32_t)((i >> 1) - 1) & 1, a.err, 5, wl)) {
                    ok = false;
                    break;
                }
                tc_fence_after();
                const uint32_t d = tmem + (uint32_t)(buf * F8_BN);
                for (int kb = 0; kb < ksteps; ++kb, ++g) {
                    const int s = (int)(g % F8_STAGES);
                    if (!mbar_wait(full0 + 8 * s, (uint32_t)(g / F8_STAGES) & 1, a.err, 3, wl)) {
                        ok = false;
                        break;
                    }
                    tc_fence_after();
                    const uint32_t sa = base + s * F8_STAGE, sb = sa + F8_A_BYTES;
#pragma unroll
                    for (int kk = 0; kk < 4; ++kk) {
                        // 32 reduction elements per MMA: +32 bytes along a K-major row, or +32 rows of
                        // the MN-major kernel tile (whose two 128-column halves are 16 KB apart)
                        const uint64_t bd = ADJ ? sdesc(sb + kk * 4096, F8_B_BYTES / 2, 1024)
                                                : sdesc(sb + kk * 32, 16, 1024);
                        umma_f8(d, sdesc(sa + kk * 32, 16, 1024), bd, idesc, (kb | kk) != 0 ? 1u : 0u);
                    }
                    umma_commit(empty0 + 8 * s);
                }
                umma_commit(accf0 + 8 * buf);
            }
            // drain: every MMA this thread issued has completed before TMEM is freed
            umma_commit(drain0);
            mbar_wait(drain0, 0, a.err, 9, TC_DRAIN_NS);
        }
    } else {
        const int q = warp & 3, half = (warp - 2) >> 2;       // lane quarter, column half
        const int ht = (warp - 2 - 4 * half) * 32 + lane;     // 0..127 within the half
        const int R = 2 * a.ncol;
        float* st = stg + half * (TC_BM * F8_LD);
        float* rowp = st + (q * 32 + lane) * F8_LD;
        long i = 0;
        for (int tile = t_first; tile < n_tiles; tile += t_stride, ++i) {
            const int k = tile / n_tiles_n, n0 = (tile - k * n_tiles_n) * F8_BN;
            const int buf = (int)(i & 1);
            if (!epilogue_all(mbar_wait(accf0 + 8 * buf, (uint32_t)(i >> 1) & 1, a.err, 4, wl))) break;
            tc_fence_after();
            const uint32_t taddr = tmem + ((uint32_t)(q * 32) << 16) + (uint32_t)(buf * F8_BN + half * 128);
            const float* isg = a.inv_sigma + (size_t)k * a.ncol;
            const float* gsk = ADJ ? nullptr : a.gscale + (size_t)k * a.nr;
#pragma unroll 1
            for (int c0 = 0; c0 < 128; c0 += 16) {
                uint32_t v[16];
                tmem_ld16(taddr + c0, v);
#pragma unroll
                for (int j = 0; j < 16; ++j) rowp[j] = __uint_as_float(v[j]);
                asm volatile("bar.sync %0, 128;" ::"r"(3 + half) : "memory");
                if (!ADJ) {
                    for (int idx = ht; idx < a.ncol * 16; idx += 128) {
                        const int n = idx % a.ncol, c = idx / a.ncol;
                        const int r = n0 + half * 128 + c0 + c;
                        const float* p0 = st + (2 * n) * F8_LD + c;           // term 0, real row 2n
                        const float re = p0[0] + 0.0625f * p0[R * F8_LD] + 0.00390625f * p0[2 * R * F8_LD];
                        const float im =
                            p0[F8_LD] + 0.0625f * p0[(R + 1) * F8_LD] + 0.00390625f * p0[(2 * R + 1) * F8_LD];
                        if (r < a.nout && MDC_INB(((size_t)k * a.nout + r) * a.ldo + a.voff_o + n, 1,
                                                  (long long)a.nf * a.nout * a.ldo, a.err, 134)) {
                            const float f = gsk[r] * isg[n];
                            a.out[((size_t)k * a.nout + r) * a.ldo + a.voff_o + n] = make_float2(re * f, im * f);
                        }
                    }
                } else {
                    // chunk columns 2j, 2j + 1 are the interleaved parts of output row s = (n0 + ...) / 2 + j
                    for (int idx = ht; idx < a.ncol * 8; idx += 128) {
                        const int n = idx % a.ncol, j = idx / a.ncol;
                        const int so = (n0 + half * 128 + c0) / 2 + j;
                        float re = 0.f, im = 0.f;
#pragma unroll
                        for (int t = F8_TERMS - 1; t >= 0; --t) {
                            const float* p0 = st + (t * R + 2 * n) * F8_LD + 2 * j;
                            const float w = t == 0 ? 1.f : (t == 1 ? 0.0625f : 0.00390625f);
                            re += w * (p0[0] + p0[F8_LD + 1]);
                            im += w * (p0[F8_LD] - p0[1]);
                        }
                        if (so < a.nout && MDC_INB(((size_t)k * a.nout + so) * a.ldo + a.voff_o + n, 1,
                                                   (long long)a.nf * a.nout * a.ldo, a.err, 135)) {
                            const float f = isg[n];
                            a.out[((size_t)k * a.nout + so) * a.ldo + a.voff_o + n] = make_float2(re * f, im * f);
                        }
                    }
                }
                asm volatile("bar.sync %0, 128;" ::"r"(3 + half) : "memory");
            }
            tc_fence_before();
            mbar_arrive(acce0 + 8 * buf);
        }
    }
    tc_fence_before();
    __syncthreads();
    if (warp == 0) {
        tc_fence_after();
        tmem_dealloc(tmem, 2 * F8_BN);
    }
}

// ------------------------------------------------------------------ B-operand preparation
template <typename T> __device__ __forceinline__ T cvt(float x);
template <> __device__ __forceinline__ __half cvt<__half>(float x) { return __float2half_rn(x); }
template <> __device__ __forceinline__ __nv_bfloat16 cvt<__nv_bfloat16>(float x) { return __float2bfloat16_rn(x); }

// Power of two with maxabs * scale < 2^emax (14 for the 16-bit operands, 8 for E4M3 terms).
__device__ __forceinline__ float pow2_scale(float maxabs, int emax) {
    if (!(maxabs > 0.f) || !isfinite(maxabs)) return 1.f;
    int e;
    frexpf(maxabs, &e);           // maxabs < 2^e
    e = e < -100 ? -100 : e;      // scale and reciprocal stay normal floats
    return ldexpf(1.f, emax - e);
}

// Packed pair of 16-bit values (lo element first in memory).
template <typename T> struct Pair2;
template <> struct Pair2<__half> {
    using type = __half2;
    static __device__ __forceinline__ __half2 make(__half a, __half b) { return __halves2half2(a, b); }
};
template <> struct Pair2<__nv_bfloat16> {
    using type = __nv_bfloat162;
    static __device__ __forceinline__ __nv_bfloat162 make(__nv_bfloat16 a, __nv_bfloat16 b) {
        return __halves2bfloat162(a, b);
    }
};

constexpr int PREP_COLS = 8;      // complex columns per CTA
constexpr int PREP_ROWS = 256;    // spatial rows per staged block (one per thread)

// Column maxima of |Re|, |Im| over the rows of a [rows][ldi] complex block (8 columns per CTA,
// each warp reading 4 rows x 64 contiguous bytes), optionally weighted per row; writes the
// power-of-two scale of each column to sig[] and its reciprocal to inv_sigma.
__device__ __forceinline__ void prep_scales(const float2* __restrict__ Xk, int ldi, int nrows, int n0, int ncol,
                                            const float* __restrict__ rw, float* red, float* sig,
                                            float* __restrict__ inv_sigma_k, int emax = 14) {
    const int j0 = threadIdx.x & 7;
    float m = 0.f;
    if (n0 + j0 < ncol) {
        // eight rows in flight per thread
        constexpr int U = 8;
        float mu[U];
#pragma unroll
        for (int u = 0; u < U; ++u) mu[u] = 0.f;
        int s = threadIdx.x >> 3;
        for (; s + 32 * (U - 1) < nrows; s += 32 * U) {
            float2 v[U];
#pragma unroll
            for (int u = 0; u < U; ++u) v[u] = Xk[(size_t)(s + 32 * u) * ldi + n0 + j0];
#pragma unroll
            for (int u = 0; u < U; ++u) {
                const float w = rw ? rw[s + 32 * u] : 1.f;
                mu[u] = fmaxf(mu[u], fmaxf(fabsf(v[u].x), fabsf(v[u].y)) * w);
            }
        }
        for (; s < nrows; s += 32) {
            const float2 v = Xk[(size_t)s * ldi + n0 + j0];
            const float w = rw ? rw[s] : 1.f;
            mu[0] = fmaxf(mu[0], fmaxf(fabsf(v.x), fabsf(v.y)) * w);
        }
#pragma unroll
        for (int u = 0; u < U; ++u) m = fmaxf(m, mu[u]);
    }
    red[threadIdx.x] = m;
    __syncthreads();
    if (threadIdx.x < PREP_COLS) {
        float mm = 0.f;
        for (int i = threadIdx.x; i < 256; i += PREP_COLS) mm = fmaxf(mm, red[i]);
        const float sc = pow2_scale(mm, emax);
        sig[threadIdx.x] = sc;
        if (n0 + (int)threadIdx.x < ncol) inv_sigma_k[n0 + threadIdx.x] = 1.f / sc;
    }
    __syncthreads();
}

// Rows [s0, s0 + 256) x 8 columns of a complex block, staged through shared memory: prep_load
// reads this thread's eight values (coalesced; rows or columns outside the block read as zero)
// and their row weights into registers, prep_put scales them by sig[column] * rw[row] into the
// tile.  Loading block b + 1 while block b is written out keeps reads in flight across the
// barriers.
constexpr int PREP_PER = PREP_ROWS * PREP_COLS / 256;
__device__ __forceinline__ void prep_load(const float2* __restrict__ Xk, int ldi, int nrows, int s0, int n0,
                                          int ncol, const float* __restrict__ rw, float2 (&v)[PREP_PER],
                                          float (&w)[PREP_PER]) {
#pragma unroll
    for (int u = 0; u < PREP_PER; ++u) {
        const int idx = threadIdx.x + 256 * u;
        const int rr = idx >> 3, j = idx & 7, s = s0 + rr;
        v[u] = make_float2(0.f, 0.f);
        w[u] = 1.f;
        if (s < nrows && n0 + j < ncol) {
            v[u] = Xk[(size_t)s * ldi + n0 + j];
            if (rw) w[u] = rw[s];
        }
    }
}
__device__ __forceinline__ void prep_put(const float2 (&v)[PREP_PER], const float (&w)[PREP_PER], const float* sig,
                                         float2 (*tile)[PREP_COLS + 1]) {
#pragma unroll
    for (int u = 0; u < PREP_PER; ++u) {
        const int idx = threadIdx.x + 256 * u;
        const int rr = idx >> 3, j = idx & 7;
        const float f = sig[j] * w[u];
        tile[rr][j] = make_float2(v[u].x * f, v[u].y * f);
    }
}

// forward: X[k][s][ldi] (voff, ncol columns) -> BT[k][n'][2*ldg], inv_sigma[k][n].  Real rows
// 2n and 2n + 1 of B hold (Re, -Im) and (Im, Re) pairs of column n along s, so the real GEMM
// over K = 2 * ldg gives the real and imaginary parts of the complex product.
template <typename T, bool SPLIT>
__global__ void __launch_bounds__(256) tc_prep_fwd(const float2* __restrict__ X, int ldi, int voff, int ns,
                                                   int ncol, int ldg, int rows_pad, T* __restrict__ BT,
                                                   float* __restrict__ inv_sigma, const int* active, size_t plane,
                                                   int* err) {
    if (active && *active == 0) return;
    using P2 = typename Pair2<T>::type;
    const int k = blockIdx.y, n0 = blockIdx.x * PREP_COLS;
    const float2* Xk = X + (size_t)k * ns * ldi + voff;
    __shared__ float red[256];
    __shared__ float sig[PREP_COLS];
    __shared__ float2 tile[PREP_ROWS][PREP_COLS + 1];
    float2 pv[PREP_PER];
    float pw[PREP_PER];
    prep_load(Xk, ldi, ns, 0, n0, ncol, nullptr, pv, pw);      // first block in flight during the scales
    prep_scales(Xk, ldi, ns, n0, ncol, nullptr, red, sig, inv_sigma + (size_t)k * ncol);
    const size_t kp = 2 * (size_t)ldg;
    P2* Bk = reinterpret_cast<P2*>(BT + (size_t)k * rows_pad * kp);      // one pair per s
    const size_t kp2 = kp / 2, plane2 = plane / 2;
    for (int s0 = 0; s0 < ldg; s0 += PREP_ROWS) {
        prep_put(pv, pw, sig, tile);
        __syncthreads();
        if (s0 + PREP_ROWS < ldg) prep_load(Xk, ldi, ns, s0 + PREP_ROWS, n0, ncol, nullptr, pv, pw);
        const int s = s0 + threadIdx.x;
        if (s < ldg) {
#pragma unroll
            for (int j = 0; j < PREP_COLS; ++j) {
                const int n = n0 + j;
                if (2 * n >= rows_pad) break;
                const float2 v = tile[threadIdx.x][j];
                const T hx = cvt<T>(v.x), hy = cvt<T>(v.y);
                if (!MDC_INB((size_t)k * rows_pad * kp2 + (size_t)(2 * n) * kp2 + s, kp2 + 1, plane2, err, 136)) break;
                P2* r0 = Bk + (size_t)(2 * n) * kp2 + s;
                r0[0] = Pair2<T>::make(hx, cvt<T>(-v.y));
                r0[kp2] = Pair2<T>::make(hy, hx);
                if (SPLIT) {
                    const float lx = v.x - (float)hx, ly = v.y - (float)hy;
                    const T tlx = cvt<T>(lx), tly = cvt<T>(ly);
                    r0[plane2] = Pair2<T>::make(tlx, cvt<T>(-ly));
                    r0[plane2 + kp2] = Pair2<T>::make(tly, tlx);
                }
            }
        }
        __syncthreads();
    }
}

// Exact split of v (|v| < 2^8) into three E4M3 terms v = h0 + h1 / 16 + h2 / 256 + e, each term the
// nearest E4M3 value of the scaled remainder (|e| <= 2^-12 |v| for normal values; the remainders are
// exact in float32).
__device__ __forceinline__ void e4m3_split3(float v, uint32_t (&h)[3]) {
    float r = v;
#pragma unroll
    for (int t = 0; t < 3; ++t) {
        const __nv_fp8_storage_t q = __nv_cvt_float_to_fp8(r, __NV_SATFINITE, __NV_E4M3);
        h[t] = q;
        const float back = __half2float(__half(__nv_cvt_fp8_to_halfraw(q, __NV_E4M3)));
        r = (r - back) * 16.f;
    }
}

// forward, E4M3 operands swapped: X[k][s][ldi] (voff, ncol columns) -> A[k][t * R + row][2 * ldg]
// bytes (R = 2 ncol; row 2n: (Re, -Im), row 2n + 1: (Im, Re) of column n along s, split into the
// three terms t of e4m3_split3 after the power-of-two column scale), inv_sigma[k][n].
__global__ void __launch_bounds__(256) tc_prep_fwd_f8(const float2* __restrict__ X, int ldi, int voff, int ns,
                                                      int ncol, int ldg, uint8_t* __restrict__ A,
                                                      float* __restrict__ inv_sigma, const int* active, int* err) {
    if (active && *active == 0) return;
    const int k = blockIdx.y, n0 = blockIdx.x * PREP_COLS;
    const float2* Xk = X + (size_t)k * ns * ldi + voff;
    __shared__ float red[256];
    __shared__ float sig[PREP_COLS];
    __shared__ float2 tile[PREP_ROWS][PREP_COLS + 1];
    float2 pv[PREP_PER];
    float pw[PREP_PER];
    prep_load(Xk, ldi, ns, 0, n0, ncol, nullptr, pv, pw);
    prep_scales(Xk, ldi, ns, n0, ncol, nullptr, red, sig, inv_sigma + (size_t)k * ncol, 8);
    const int R = 2 * ncol;
    const size_t kp = 2 * (size_t)ldg;
    uint16_t* Ak = reinterpret_cast<uint16_t*>(A + (size_t)k * F8_TERMS * R * kp);   // two bytes per s
    const size_t row2 = kp / 2;
    for (int s0 = 0; s0 < ldg; s0 += PREP_ROWS) {
        prep_put(pv, pw, sig, tile);
        __syncthreads();
        if (s0 + PREP_ROWS < ldg) prep_load(Xk, ldi, ns, s0 + PREP_ROWS, n0, ncol, nullptr, pv, pw);
        const int s = s0 + threadIdx.x;
        if (s < ldg) {
#pragma unroll
            for (int j = 0; j < PREP_COLS; ++j) {
                const int n = n0 + j;
                if (n >= ncol) break;
                const float2 v = tile[threadIdx.x][j];
                uint32_t hx[3], hy[3], hny[3];
                e4m3_split3(v.x, hx);
                e4m3_split3(v.y, hy);
                e4m3_split3(-v.y, hny);
#pragma unroll
                for (int t = 0; t < F8_TERMS; ++t) {
                    if (!MDC_INB((size_t)k * F8_TERMS * R * row2 + (size_t)(t * R + 2 * n) * row2 + s, row2 + 1,
                                 (long long)gridDim.y * F8_TERMS * R * row2, err, 138))
                        continue;
                    uint16_t* r0 = Ak + (size_t)(t * R + 2 * n) * row2 + s;
                    r0[0] = (uint16_t)(hx[t] | (hny[t] << 8));          // (Re, -Im)
                    r0[row2] = (uint16_t)(hy[t] | (hx[t] << 8));        // (Im, Re)
                }
            }
        }
        __syncthreads();
    }
}

// adjoint, E4M3 operands swapped: Y[k][r][ldi] (voff, ncol columns) * gscale[k][r] ->
// A[k][t * R + row][kpitch] bytes (row 2n: Re, 2n + 1: Im of column n along r, split into the three
// terms t of e4m3_split3 after the power-of-two column scale; zero for r >= nr), inv_sigma[k][n].
__global__ void __launch_bounds__(256) tc_prep_adj_f8(const float2* __restrict__ Y, int ldi, int voff, int nr,
                                                      int ncol, const float* __restrict__ gscale, int kpitch,
                                                      uint8_t* __restrict__ A, float* __restrict__ inv_sigma,
                                                      const int* active, int* err) {
    if (active && *active == 0) return;
    const int k = blockIdx.y, n0 = blockIdx.x * PREP_COLS;
    const float2* Yk = Y + (size_t)k * nr * ldi + voff;
    const float* gs = gscale + (size_t)k * nr;
    __shared__ float red[256];
    __shared__ float sig[PREP_COLS];
    __shared__ float2 tile[PREP_ROWS][PREP_COLS + 1];
    float2 pv[PREP_PER];
    float pw[PREP_PER];
    prep_load(Yk, ldi, nr, 0, n0, ncol, gs, pv, pw);
    prep_scales(Yk, ldi, nr, n0, ncol, gs, red, sig, inv_sigma + (size_t)k * ncol, 8);
    const int R = 2 * ncol;
    uint16_t* Ak = reinterpret_cast<uint16_t*>(A + (size_t)k * F8_TERMS * R * kpitch);   // two bytes per r pair
    const size_t kq = (size_t)kpitch / 2;
    for (int r0 = 0; r0 < kpitch; r0 += PREP_ROWS) {
        prep_put(pv, pw, sig, tile);
        __syncthreads();
        if (r0 + PREP_ROWS < kpitch) prep_load(Yk, ldi, nr, r0 + PREP_ROWS, n0, ncol, gs, pv, pw);
        // threads 0..127 each take rows r0 + 2t, r0 + 2t + 1 for columns 0..3, threads 128..255 columns 4..7
        const int t = threadIdx.x & 127, jb = (threadIdx.x >> 7) * (PREP_COLS / 2);
        const int r = r0 + 2 * t;
        if (r < kpitch) {
#pragma unroll
            for (int jj = 0; jj < PREP_COLS / 2; ++jj) {
                const int j = jb + jj, n = n0 + j;
                if (n >= ncol) continue;
                const float2 va = tile[2 * t][j], vb = tile[2 * t + 1][j];
                uint32_t ax[3], bx[3], ay[3], by[3];
                e4m3_split3(va.x, ax);
                e4m3_split3(vb.x, bx);
                e4m3_split3(va.y, ay);
                e4m3_split3(vb.y, by);
#pragma unroll
                for (int tt = 0; tt < F8_TERMS; ++tt) {
                    if (!MDC_INB((size_t)k * F8_TERMS * R * kq + (size_t)(tt * R + 2 * n) * kq + (r >> 1), kq + 1,
                                 (long long)gridDim.y * F8_TERMS * R * kq, err, 139))
                        continue;
                    uint16_t* q0 = Ak + (size_t)(tt * R + 2 * n) * kq + (r >> 1);
                    q0[0] = (uint16_t)(ax[tt] | (bx[tt] << 8));           // Re at r, r + 1
                    q0[kq] = (uint16_t)(ay[tt] | (by[tt] << 8));          // Im at r, r + 1
                }
            }
        }
        __syncthreads();
    }
}

// adjoint: Y[k][r][ldi] (voff, ncol columns) * gscale[k][r] -> BT[k][n''][kpitch], inv_sigma[k][n].
// Real rows 2n and 2n + 1 hold Re and Im of column n along r; each thread writes two adjacent r.
template <typename T, bool SPLIT>
__global__ void __launch_bounds__(256) tc_prep_adj(const float2* __restrict__ Y, int ldi, int voff, int nr,
                                                   int ncol, const float* __restrict__ gscale, int kpitch,
                                                   int rows_pad, T* __restrict__ BT, float* __restrict__ inv_sigma,
                                                   const int* active, size_t plane, int* err) {
    if (active && *active == 0) return;
    using P2 = typename Pair2<T>::type;
    const int k = blockIdx.y, n0 = blockIdx.x * PREP_COLS;
    const float2* Yk = Y + (size_t)k * nr * ldi + voff;
    const float* gs = gscale + (size_t)k * nr;
    __shared__ float red[256];
    __shared__ float sig[PREP_COLS];
    __shared__ float2 tile[PREP_ROWS][PREP_COLS + 1];
    float2 pv[PREP_PER];
    float pw[PREP_PER];
    prep_load(Yk, ldi, nr, 0, n0, ncol, gs, pv, pw);            // first block in flight during the scales
    prep_scales(Yk, ldi, nr, n0, ncol, gs, red, sig, inv_sigma + (size_t)k * ncol);
    P2* Bk = reinterpret_cast<P2*>(BT + (size_t)k * rows_pad * kpitch);  // kpitch is a multiple of 8
    const size_t kq = (size_t)kpitch / 2, plane2 = plane / 2;
    for (int r0 = 0; r0 < kpitch; r0 += PREP_ROWS) {
        prep_put(pv, pw, sig, tile);
        __syncthreads();
        if (r0 + PREP_ROWS < kpitch) prep_load(Yk, ldi, nr, r0 + PREP_ROWS, n0, ncol, gs, pv, pw);
        // threads 0..127 each take rows r0 + 2t, r0 + 2t + 1 for columns 0..3, threads 128..255 columns 4..7
        const int t = threadIdx.x & 127, jb = (threadIdx.x >> 7) * (PREP_COLS / 2);
        const int r = r0 + 2 * t;
        if (r < kpitch) {
#pragma unroll
            for (int jj = 0; jj < PREP_COLS / 2; ++jj) {
                const int j = jb + jj, n = n0 + j;
                if (2 * n >= rows_pad) continue;
                const float2 a = tile[2 * t][j], b = tile[2 * t + 1][j];
                const T ax = cvt<T>(a.x), bx = cvt<T>(b.x), ay = cvt<T>(a.y), by = cvt<T>(b.y);
                if (!MDC_INB((size_t)k * rows_pad * kq + (size_t)(2 * n) * kq + (r >> 1), kq + 1, plane2, err, 137)) continue;
                P2* q0 = Bk + (size_t)(2 * n) * kq + (r >> 1);
                q0[0] = Pair2<T>::make(ax, bx);
                q0[kq] = Pair2<T>::make(ay, by);
                if (SPLIT) {
                    q0[plane2] = Pair2<T>::make(cvt<T>(a.x - (float)ax), cvt<T>(b.x - (float)bx));
                    q0[plane2 + kq] = Pair2<T>::make(cvt<T>(a.y - (float)ay), cvt<T>(b.y - (float)by));
                }
            }
        }
        __syncthreads();
    }
}

// ------------------------------------------------------------------ host side
PFN_cuTensorMapEncodeTiled_v12000 encode_fn() {
    static PFN_cuTensorMapEncodeTiled_v12000 fn = nullptr;
    if (!fn) {
        void* p = nullptr;
        cudaDriverEntryPointQueryResult q;
        if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", &p, 12000, cudaEnableDefault, &q) ==
                cudaSuccess &&
            q == cudaDriverEntryPointSuccess)
            fn = reinterpret_cast<PFN_cuTensorMapEncodeTiled_v12000>(p);
    }
    return fn;
}

bool make_map_3d(CUtensorMap* m, const void* ptr, bool bf16, uint64_t d0, uint64_t d1, uint64_t d2,
                 uint64_t pitch1_bytes, uint64_t pitch2_bytes, uint32_t b0, uint32_t b1, bool bytes = false,
                 bool byte_swizzle = false) {
    auto enc = encode_fn();
    if (!enc) return false;
    // E4M3 bytes move as 4-byte elements (four values each): d0 and b0 are given in bytes
    cuuint64_t dims[3] = {bytes ? d0 / 4 : d0, d1, d2};
    cuuint64_t strides[2] = {pitch1_bytes, pitch2_bytes};
    cuuint32_t box[3] = {bytes ? b0 / 4 : b0, b1, 1};
    cuuint32_t es[3] = {1, 1, 1};
    // 16-bit operands land 128-byte swizzled for the MMA; E4M3 bytes land unswizzled for widening in
    // shared memory, or 128-byte swizzled for the row-per-lane widening into tensor memory
    const CUtensorMapDataType dt = bytes ? CU_TENSOR_MAP_DATA_TYPE_UINT32
                                         : (bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT16);
    CUresult r = enc(m, dt, 3, const_cast<void*>(ptr), dims, strides, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE,
                     (bytes && !byte_swizzle) ? CU_TENSOR_MAP_SWIZZLE_NONE : CU_TENSOR_MAP_SWIZZLE_128B,
                     CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE);
    return r == CUDA_SUCCESS;
}

int pick_bn(int n2) {
    if (n2 <= 32) return 32;
    if (n2 <= 64) return 64;
    if (n2 <= 128) return 128;
    return 256;
}

// SMs of the current device (queried per call: a process may drive several devices)
int sm_count() {
    int dev = 0, n = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&n, cudaDevAttrMultiProcessorCount, dev);
    return n > 0 ? n : 148;
}

// grid: (column tiles, row tiles, frequencies), walked by min(tiles, SMs) persistent CTAs.
template <bool ADJ, int BN, bool SPLIT, bool CVT = false>
bool launch_tc(const CUtensorMap* maps, const TcArgs& a, uint32_t idesc, dim3 grid, cudaStream_t s,
               const int* active) {
    static SmemLimit attr;
    const size_t smem = tc_smem_bytes<BN, SPLIT, CVT, ADJ>();
    constexpr int THREADS = CVT ? TC_THREADS + TC_CVT_THREADS + 32 : TC_THREADS;
    auto kern = tc_gemm_kernel<ADJ, BN, SPLIT, CVT>;
    attr.ensure(kern, (int)smem);
    const int n_tiles = (int)grid.x * (int)grid.y * (int)grid.z;
    const int ctas = n_tiles < sm_count() ? n_tiles : sm_count();
    kern<<<ctas, THREADS, smem, s>>>(maps[0], maps[1], maps[2], maps[3], a, idesc, active, (int)grid.x,
                                     (int)grid.y, n_tiles);
    return true;
}

// MDC_E4M3_SWAP=0 in the environment keeps narrow E4M3 forward products on the widening kernel
// (for comparisons).
bool f8_swap_allowed() {
    static int env = -1;
    if (env < 0) {
        const char* e = getenv("MDC_E4M3_SWAP");
        env = (e && e[0] == '0') ? 0 : 1;
    }
    return env == 1;
}

}  // namespace

int tc_rows_pad(int ncol) {
    const int n2 = 2 * ncol;
    const int bn = pick_bn(n2);
    return (n2 + bn - 1) / bn * bn;
}

size_t tc_scratch_elems(const mdc_plan* p, int ncol) {
    size_t rows = (size_t)tc_rows_pad(ncol);
    // E4M3 forward products of few columns take three byte rows per real row (2 ncol real rows):
    // 6 ncol bytes = 3 ncol 16-bit elements per reduction element
    if (p->storage == MDC_CE4M3 && 3 * (size_t)ncol > rows) rows = 3 * (size_t)ncol;
    const size_t kfwd = 2 * (size_t)p->ldg;
    const size_t kadj = (size_t)round_up(p->nr, p->storage == MDC_CE4M3 ? 16 : 8);
    return (size_t)p->nf * rows * (kfwd > kadj ? kfwd : kadj);
}

bool tc_supported(const mdc_plan* p, int ncol) {
    return storage_tc(p->storage) && (ncol >= 8 || p->force_tc) && p->tcB != nullptr && ncol <= p->tc_cap &&
           encode_fn() != nullptr;
}

// Per-frequency product on tensor cores; returns false if it could not be launched.
bool launch_tc_product(mdc_plan* p, bool adjoint, const float2* in, int ldi, int voff_i, float2* out, int ldo,
                       int voff_o, int ncol, cudaStream_t s, const int* active, int bn_override, bool scoped) {
    const bool bf16 = p->storage == MDC_CBF16;
    const bool split = p->storage == MDC_C32S;
    const bool e4m3 = p->storage == MDC_CE4M3;      // bytes widened to FP16 in shared memory
    int bn = bn_override ? bn_override : pick_bn(2 * ncol);
    if (split && bn > 128) bn = 128;   // the split epilogue keeps a BN-wide float32 row in registers
    if (bn != 32 && bn != 64 && bn != 128 && bn != 256) return false;
    const int rows_pad = (2 * ncol + bn - 1) / bn * bn;
    if (rows_pad > tc_rows_pad(p->tc_cap)) return false;
    const int kpitch = (int)round_up(p->nr, 8);
    const uint64_t kp = 2 * (uint64_t)p->ldg;
    // B operand (and its lo half for the split format, one plane further)
    const size_t plane = (size_t)p->nf * rows_pad * (adjoint ? (size_t)kpitch : (size_t)kp);
    dim3 pg((unsigned)(rows_pad / 16), (unsigned)p->nf);
    std::optional<LaunchScope> scope;
    if (e4m3 && !bn_override && ncol <= F8_MAX_COLS && f8_swap_allowed()) {
        // operands swapped: spectra split into three E4M3 terms, kernel bytes as the wide operand
        const int arows = F8_TERMS * 2 * ncol;
        const uint64_t kpf = (uint64_t)round_up(p->nr, 16);     // adjoint reduction pitch (bytes)
        if (scoped) scope.emplace(p, s, MDC_KC_TC_PREP);
        dim3 pf((unsigned)((ncol + PREP_COLS - 1) / PREP_COLS), (unsigned)p->nf);
        if (!adjoint)
            tc_prep_fwd_f8<<<pf, 256, 0, s>>>(in, ldi, voff_i, p->ns, ncol, (int)p->ldg, (uint8_t*)p->tcB,
                                              p->tcSigma, active, p->err_flag);
        else
            tc_prep_adj_f8<<<pf, 256, 0, s>>>(in, ldi, voff_i, p->nr, ncol, p->gscale, (int)kpf, (uint8_t*)p->tcB,
                                              p->tcSigma, active, p->err_flag);
        scope.reset();
        CUtensorMap mA, mB;
        const uint64_t ka = adjoint ? kpf : kp;
        if (!make_map_3d(&mA, p->tcB, false, ka, (uint64_t)arows, p->nf, ka, ka * arows, 128, TC_BM, true, true) ||
            !make_map_3d(&mB, p->G, false, kp, p->nr, p->nf, kp, kp * p->nr, 128, adjoint ? 128 : F8_BN, true, true))
            return false;
        TcArgs a{};
        a.nf = p->nf;
        a.kstages = adjoint ? (p->nr + 127) / 128 : (int)(kp / 128);
        a.nout = adjoint ? p->ns : p->nr;
        a.nr = p->nr;
        a.ncol = ncol;
        a.inv_sigma = p->tcSigma;
        a.gscale = p->gscale;
        a.out = out;
        a.ldo = ldo;
        a.voff_o = voff_o;
        a.err = p->err_flag;
        a.wait_ns = p->wait_ns;
        // kind::f8f6f4: D float32, A and B E4M3 (format 0), A K-major, B K-major (forward) or
        // MN-major (adjoint), N = 256, M = 128
        const uint32_t idesc = (1u << 4) | ((adjoint ? 1u : 0u) << 16) | ((uint32_t)(F8_BN >> 3) << 17) |
                               ((uint32_t)(TC_BM >> 4) << 24);
        const int ntn = adjoint ? (int)((kp + F8_BN - 1) / F8_BN) : (p->nr + F8_BN - 1) / F8_BN;
        const int n_tiles = ntn * p->nf;
        const size_t smem = f8_smem_bytes();
        const int ctas = n_tiles < sm_count() ? n_tiles : sm_count();
        if (scoped) scope.emplace(p, s, adjoint ? MDC_KC_PRODUCT_ADJ : MDC_KC_PRODUCT_FWD);
        if (!adjoint) {
            static SmemLimit attr;
            attr.ensure(tc_f8_kernel<false>, (int)smem);
            tc_f8_kernel<false><<<ctas, TC_THREADS, smem, s>>>(mA, mB, a, idesc, active, ntn, n_tiles);
        } else {
            static SmemLimit attr;
            attr.ensure(tc_f8_kernel<true>, (int)smem);
            tc_f8_kernel<true><<<ctas, TC_THREADS, smem, s>>>(mA, mB, a, idesc, active, ntn, n_tiles);
        }
        return true;
    }
    if (scoped) scope.emplace(p, s, MDC_KC_TC_PREP);
#define MDC_PREP(KER, T, SP, ...) KER<T, SP><<<pg, 256, 0, s>>>(__VA_ARGS__, active, plane, p->err_flag)
    if (!adjoint) {
        if (bf16)
            MDC_PREP(tc_prep_fwd, __nv_bfloat16, false, in, ldi, voff_i, p->ns, ncol, (int)p->ldg, rows_pad,
                     (__nv_bfloat16*)p->tcB, p->tcSigma);
        else if (split)
            MDC_PREP(tc_prep_fwd, __half, true, in, ldi, voff_i, p->ns, ncol, (int)p->ldg, rows_pad,
                     (__half*)p->tcB, p->tcSigma);
        else
            MDC_PREP(tc_prep_fwd, __half, false, in, ldi, voff_i, p->ns, ncol, (int)p->ldg, rows_pad,
                     (__half*)p->tcB, p->tcSigma);
    } else {
        if (bf16)
            MDC_PREP(tc_prep_adj, __nv_bfloat16, false, in, ldi, voff_i, p->nr, ncol, p->gscale, kpitch, rows_pad,
                     (__nv_bfloat16*)p->tcB, p->tcSigma);
        else if (split)
            MDC_PREP(tc_prep_adj, __half, true, in, ldi, voff_i, p->nr, ncol, p->gscale, kpitch, rows_pad,
                     (__half*)p->tcB, p->tcSigma);
        else
            MDC_PREP(tc_prep_adj, __half, false, in, ldi, voff_i, p->nr, ncol, p->gscale, kpitch, rows_pad,
                     (__half*)p->tcB, p->tcSigma);
    }
#undef MDC_PREP
    scope.reset();
    // tensor maps: A over the kernel copy [nf][nr][2*ldg] (16-bit reals), B over the prepared operand
    CUtensorMap maps[4];
    const unsigned char* G = static_cast<const unsigned char*>(p->G);
    const unsigned char* Bp = static_cast<const unsigned char*>(p->tcB);
    const size_t glo = split ? (size_t)p->nf * p->nr * p->ldg * 4 : 0;   // lo plane of the kernel
    const size_t blo = plane * 2;                                          // lo plane of B (bytes)
    // row tiles of the product (kernel rows forward; 2 * ldg interleaved reals adjoint)
    const int mrows = adjoint ? (int)(kp / TC_BM) : (p->nr + TC_BM - 1) / TC_BM;
    const int bbox = bn;
    bool ok = true;
    const uint64_t ab = e4m3 ? 1 : 2;         // bytes per real of the kernel copy
    // E4M3 byte tiles: forward 128 rows x 128 bytes for B tiles of <= 64 columns (two reduction
    // slices per stage), else 128 x 64; adjoint 128 (<= 64 columns) or 64 reduction rows x 128
    // bytes (both output-row halves)
    const int ks = tc_cvt_ksub(bn);
    const uint32_t fa0 = e4m3 ? 64 * ks : 64, aa0 = e4m3 ? 128 : 64, aa1 = e4m3 ? 64 * ks : 64;
    for (int h = 0; h < (split ? 2 : 1) && ok; ++h) {
        const void* ga = G + h * glo;
        const void* gb = Bp + h * blo;
        if (!adjoint)
            ok = make_map_3d(&maps[2 * h], ga, bf16, kp, p->nr, p->nf, kp * ab, kp * ab * p->nr, fa0, 128, e4m3,
                             e4m3 && ks == 2) &&
                 make_map_3d(&maps[2 * h + 1], gb, bf16, kp, rows_pad, p->nf, kp * 2, kp * 2 * rows_pad, 64, bbox);
        else
            ok = make_map_3d(&maps[2 * h], ga, bf16, kp, p->nr, p->nf, kp * ab, kp * ab * p->nr, aa0, aa1, e4m3) &&
                 make_map_3d(&maps[2 * h + 1], gb, bf16, p->nr, rows_pad, p->nf, (uint64_t)kpitch * 2,
                             (uint64_t)kpitch * 2 * rows_pad, 64, bbox);
    }
    if (!ok) return false;
    if (!split) {
        maps[2] = maps[0];
        maps[3] = maps[1];
    }
    TcArgs a{};
    a.nf = p->nf;
    a.kstages = adjoint ? (p->nr + TC_BK - 1) / TC_BK : (int)(kp / TC_BK);
    a.nout = adjoint ? p->ns : p->nr;
    a.nr = p->nr;
    a.ncol = ncol;
    a.inv_sigma = p->tcSigma;
    a.gscale = p->gscale;
    a.out = out;
    a.ldo = ldo;
    a.voff_o = voff_o;
    a.err = p->err_flag;
    a.wait_ns = p->wait_ns;
    const uint32_t fmt = bf16 ? 1u : 0u;
    const uint32_t idesc = (1u << 4) | (fmt << 7) | (fmt << 10) | ((adjoint ? 1u : 0u) << 15) |
                           ((uint32_t)(bn >> 3) << 17) | ((uint32_t)(TC_BM >> 4) << 24);
    dim3 grid((unsigned)(rows_pad / bn), (unsigned)mrows, (unsigned)p->nf);
    if (scoped) scope.emplace(p, s, adjoint ? MDC_KC_PRODUCT_ADJ : MDC_KC_PRODUCT_FWD);
#define MDC_TC_LAUNCH(ADJV, BV, SPV)                                                             \
    if (e4m3)                                                                                    \
        launched = launch_tc<ADJV, BV, false, true>(maps, a, idesc, grid, s, active);               \
    else                                                                                         \
        launched = launch_tc<ADJV, BV, SPV>(maps, a, idesc, grid, s, active);
#define MDC_TC_CASE(BNV)                                                                   \
    case BNV:                                                                              \
        if (split) {                                                                       \
            constexpr int BS = BNV > 128 ? 128 : BNV;                                      \
            if (adjoint) { MDC_TC_LAUNCH(true, BS, true) }                                 \
            else { MDC_TC_LAUNCH(false, BS, true) }                                        \
        } else {                                                                           \
            if (adjoint) { MDC_TC_LAUNCH(true, BNV, false) }                               \
            else { MDC_TC_LAUNCH(false, BNV, false) }                                      \
        }                                                                                  \
        break;
    bool launched = false;
    switch (bn) {
        MDC_TC_CASE(32)
        MDC_TC_CASE(64)
        MDC_TC_CASE(128)
        MDC_TC_CASE(256)
    }
#undef MDC_TC_CASE
#undef MDC_TC_LAUNCH
    return launched;
}

}  // namespace mdc
