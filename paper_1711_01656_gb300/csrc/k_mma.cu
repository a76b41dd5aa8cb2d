// k_mma.cu -- the count tiles as tensor-core products (tcgen05, sm_103a).
//
// The 2-D inclusive prefix of a tile's one-hot plane of bin b (Eq. 2.15
// inside a tile) is a product of 0/1 matrices:
//   H_local = T . O_b . T^t,   O_b[r][c] = [bin(r, c) = b],
//   T[x][y] = [y <= x]   (lower-triangular ones, 128 x 128),
// computed as two chained MMAs with fp32 accumulators in tensor memory:
//   D1 = T . O_b          (column prefix: D1[r][c] = sum_{r' <= r} O_b[r'][c])
//   D2 = D1 . T^t         (row prefix:    D2[r][c] = sum_{c' <= c} D1[r][c'])
// Operands are bf16 0/1 (and D1 <= 128, exact in bf16: 8 significant
// bits), accumulation fp32 (D2 <= 16384, exact below 2^24), so the counts are
// exact.  The 8-bit integer MMA kind is not available on sm_103a (ptxas
// refuses .kind::i8 for this target), hence .kind::f16 with bf16 operands.
// The tile's carries from the tiles above and to the left (the corner, the
// prefix over the tile's columns of the column counts above it, the prefix
// over its rows of the row counts to its left; the same carries as the
// scan-based tiles kernel, from k_tile_sums_all and k_carry_scan on a grid of
// 128 x 128 tiles) are added in the epilogue, and the tile is written once,
// bin-major, through a shared-memory stage so that every warp store covers
// a 512-byte row.
//
// One CTA of 128 threads (4 warps, one per 32 TMEM lanes) per (tile,
// channel); it loops over the channel's bins.  Shared memory holds T (the A
// operand of the first MMA and, read as N x K, the B operand of the second:
// both are [y <= x]), the one-hot O_b^t (B of the first MMA), D1 converted to
// bf16 (A of the second), the tile's bins and the output stage.  All matrix
// operands are K-major with no swizzle: 8 x 16-byte core matrices, 128 bytes
// each, 8-row groups 128 bytes apart (SBO) and 8-column groups 2048 bytes
// apart (LBO).  One elected thread issues the MMAs (K = 16 per instruction)
// and commits them to an mbarrier; every wait on it is bounded: a wait that
// gives up sets bit 2 of the context's error word (ih_sync then reports
// IH_ETIMEOUT), the CTA stops issuing work, frees its tensor memory and
// returns.
#include <stdint.h>

#include <mutex>

#include "ih_internal.cuh"

namespace ih {

namespace {

constexpr int kMT = 128;                 // tile side
constexpr int kMThreads = 128;
constexpr uint32_t kMatBytes = 128 * 128 * 2;   // one bf16 operand
constexpr uint32_t kLBO = 2048, kSBO = 128;
constexpr int kBinStride = kMT + 16;     // bytes per row of the transposed bin tile
constexpr int kOutStride = kMT + 4;      // int32 per row of the output stage
constexpr uint32_t kTmemCols = 256;      // D1 in columns 0..127, D2 in 128..255
constexpr long kWaitLimit = 1L << 24;    // mbarrier polls before giving up

struct __align__(1024) MmaSmem {
    uint8_t T[kMatBytes];                // [y <= x], K-major 128 x 128 bf16
    uint8_t OT[kMatBytes];               // O_b^t: row c, k = r
    uint8_t XA[kMatBytes];               // D1 as bf16: row r, k = c
    uint8_t binT[kMT][kBinStride];       // bin of pixel (r, c) at binT[c][r]; 0xff: none
    int32_t out[kMT][kOutStride];        // the output stage
    int32_t gp[kMT], lp[kMT];            // carries: column prefix of G, row prefix of L
    uint64_t mbar;
    uint32_t tmem_base;
    int32_t stop;
};

// Byte offset of element (row, k) of a K-major, unswizzled 128 x 128 bf16 operand.
__device__ __forceinline__ uint32_t kmaj_off(int row, int k)
{
    return (uint32_t)(k >> 3) * kLBO + (uint32_t)(row >> 3) * kSBO + (uint32_t)(row & 7) * 16 + (uint32_t)(k & 7) * 2;
}

__device__ __forceinline__ uint32_t smem_addr(const void *p) { return (uint32_t)__cvta_generic_to_shared(p); }

// Shared-memory matrix descriptor (tcgen05): start address, leading (K)
// and stride (M/N) byte offsets, all >> 4; descriptor version 1 at bit 46;
// base offset 0, relative LBO mode, no swizzle.
__device__ __forceinline__ uint64_t smem_desc(uint32_t saddr)
{
    return (uint64_t)((saddr >> 4) & 0x3FFF) | ((uint64_t)((kLBO >> 4) & 0x3FFF) << 16) |
           ((uint64_t)((kSBO >> 4) & 0x3FFF) << 32) | ((uint64_t)1 << 46);
}

// Instruction descriptor of kind::f16: D fp32 (bits 4-5 = 1), A and B bf16
// (bits 7-9 = 1, 10-12 = 1), both K-major (bits 15, 16 = 0), N >> 3 at bits
// 17-22, M >> 4 at bits 24-28.
constexpr uint32_t kIdesc = (1u << 4) | (1u << 7) | (1u << 10) | ((uint32_t)(kMT >> 3) << 17) |
                            ((uint32_t)(kMT >> 4) << 24);

__device__ __forceinline__ void mma_bf16(uint32_t d_tmem, uint64_t a, uint64_t b, uint32_t accumulate)
{
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(d_tmem),
        "l"(a), "l"(b), "r"(kIdesc), "r"(accumulate));
}

__device__ __forceinline__ void mma_commit(uint64_t *mbar)
{
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     smem_addr(mbar))
                 : "memory");
}

__device__ __forceinline__ bool mbar_try_wait(uint64_t *mbar, uint32_t parity)
{
    uint32_t ok;
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(ok)
        : "r"(smem_addr(mbar)), "r"(parity)
        : "memory");
    return ok != 0;
}

__device__ __forceinline__ void fence_before_sync() { asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_after_sync() { asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory"); }
__device__ __forceinline__ void fence_async_smem() { asm volatile("fence.proxy.async.shared::cta;" ::: "memory"); }

// 32 consecutive fp32 columns of this thread's TMEM lane.
__device__ __forceinline__ void tmem_ld32(uint32_t taddr, uint32_t (&v)[32])
{
    asm volatile(
        "tcgen05.ld.sync.aligned.32x32b.x32.b32 {%0, %1, %2, %3, %4, %5, %6, %7, %8, %9, %10, %11, %12, %13, %14, "
        "%15, %16, %17, %18, %19, %20, %21, %22, %23, %24, %25, %26, %27, %28, %29, %30, %31}, [%32];"
        : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]), "=r"(v[7]),
          "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]), "=r"(v[13]), "=r"(v[14]), "=r"(v[15]),
          "=r"(v[16]), "=r"(v[17]), "=r"(v[18]), "=r"(v[19]), "=r"(v[20]), "=r"(v[21]), "=r"(v[22]), "=r"(v[23]),
          "=r"(v[24]), "=r"(v[25]), "=r"(v[26]), "=r"(v[27]), "=r"(v[28]), "=r"(v[29]), "=r"(v[30]), "=r"(v[31])
        : "r"(taddr));
}

__device__ __forceinline__ void tmem_wait_ld() { asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory"); }

// The 8 MMAs (K = 16 each) of one 128 x 128 x 128 product D = A . B, A and B
// K-major in shared memory (B stored as N x K).
__device__ __forceinline__ void issue_product(uint32_t d_tmem, uint32_t a_saddr, uint32_t b_saddr)
{
#pragma unroll
    for (int ks = 0; ks < kMT / 16; ++ks)
        mma_bf16(d_tmem, smem_desc(a_saddr + ks * 2 * kLBO), smem_desc(b_saddr + ks * 2 * kLBO), ks > 0 ? 1u : 0u);
}

// Waits for phase `parity` of the MMA barrier; false when the bound ran out.
__device__ __forceinline__ bool wait_product(uint64_t *mbar, uint32_t parity)
{
    for (long k = 0; k < kWaitLimit; ++k)
        if (mbar_try_wait(mbar, parity)) return true;
    return false;
}

// Eq. 2.15's binning function: uniform over [0,256) or the value as the bin.
__device__ __forceinline__ int mma_bin_of(int v, int bins, int mode)
{
    if (mode == 0) return (v * bins) >> 8;
    return v < bins ? v : -1;
}

// bf16 1.0 in the low / high half of a word for one-hot pairs.
__device__ __forceinline__ uint32_t onehot2(uint32_t bins2, uint32_t b)
{
    return ((bins2 & 0xffu) == b ? 0x3F80u : 0u) | (((bins2 >> 8) & 0xffu) == b ? 0x3F800000u : 0u);
}

__global__ void __launch_bounds__(kMThreads, 1) k_tiles_mma(const __grid_constant__ PlaneSet ps, int *err)
{
    extern __shared__ unsigned char dsm_raw[];
    MmaSmem &sm = *reinterpret_cast<MmaSmem *>((reinterpret_cast<uintptr_t>(dsm_raw) + 1023) & ~uintptr_t(1023));
    pdl_wait();
    const TileGrid &g = ps.g;
    const int j = blockIdx.x, i = blockIdx.y;
    const ChanDev &cd = ps.chan[blockIdx.z];
    const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
    const int R0 = i * g.R, nr = min(g.R, g.H - R0);
    const int C0 = j * g.Wc, nc = min(kMT, g.W - C0);

    // T = [y <= x] as 16-byte chunks (row x, columns 8kg .. 8kg + 7)
    for (int k = tid; k < kMT * (kMT / 8); k += kMThreads) {
        const int x = k >> 4, kg = k & 15;
        uint32_t w[4];
#pragma unroll
        for (int q = 0; q < 4; ++q) {
            const int y0 = kg * 8 + 2 * q;
            w[q] = (y0 <= x ? 0x3F80u : 0u) | (y0 + 1 <= x ? 0x3F800000u : 0u);
        }
        *reinterpret_cast<uint4 *>(sm.T + kmaj_off(x, kg * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
    }
    // the tile's bins, transposed (0xff outside the frame and for values in no bin)
    for (int k = tid; k < kMT * kMT; k += kMThreads) {
        const int r = k >> 7, c = k & 127;
        int q = -1;
        if (r < nr && c < nc) q = mma_bin_of(__ldg(cd.plane + (int64_t)(R0 + r) * cd.pitch + C0 + c), cd.bins, cd.mode);
        sm.binT[c][r] = q < 0 ? (uint8_t)0xff : (uint8_t)q;
    }
    if (warp == 0) {
        asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(smem_addr(&sm.tmem_base)),
                     "r"(kTmemCols)
                     : "memory");
        asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;" ::: "memory");
    }
    if (tid == 0) {
        asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(smem_addr(&sm.mbar)) : "memory");
        asm volatile("fence.mbarrier_init.release.cluster;" ::: "memory");
    }
    fence_async_smem();
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    const uint32_t tmem = sm.tmem_base, d1 = tmem, d2 = tmem + kMT;
    const uint32_t lanes = (uint32_t)(warp * 32) << 16;  // this warp's quarter of the TMEM lanes
    const bool carries = ps.colsum != nullptr;
    uint32_t parity = 0;
    bool ok = true;
    __shared__ int32_t s_tr;
    for (int b = 0; b < cd.bins; ++b) {
        const int64_t gb = cd.bin_off + b;
        // O_b^t: row c, k = r (8 rows of one column per 16-byte chunk)
        for (int k = tid; k < kMT * 16; k += kMThreads) {
            const int c = k & 127, rg = k >> 7;
            const uint2 bb = *reinterpret_cast<const uint2 *>(&sm.binT[c][rg * 8]);
            *reinterpret_cast<uint4 *>(sm.OT + kmaj_off(c, rg * 8)) =
                make_uint4(onehot2(bb.x, b), onehot2(bb.x >> 16, b), onehot2(bb.y, b), onehot2(bb.y >> 16, b));
        }
        // carries of bin b: inclusive prefixes of G over the tile's columns and
        // of L over its rows, and the corner H(R0 - 1, C0 - 1)
        if (warp < 2) {
            const int n = warp == 0 ? nc : nr;
            int v[4];
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                const int x = 4 * lane + q;
                v[q] = 0;
                if (carries && x < n)
                    v[q] = warp == 0 ? ps.colsum[((int64_t)i * ps.B + gb) * g.W + C0 + x]
                                     : ps.rowsum[((int64_t)j * ps.B + gb) * g.H + R0 + x];
            }
            v[1] += v[0];
            v[2] += v[1];
            v[3] += v[2];
            int incl = v[3];
#pragma unroll
            for (int d = 1; d < 32; d <<= 1) {
                const int y = __shfl_up_sync(0xffffffffu, incl, d);
                if (lane >= d) incl += y;
            }
            int32_t *dst = warp == 0 ? sm.gp : sm.lp;
#pragma unroll
            for (int q = 0; q < 4; ++q) dst[4 * lane + q] = incl - v[3] + v[q];
        } else if (warp == 2) {
            int t = 0;
            if (carries)
                for (int ib = lane; ib < i; ib += 32) t += ps.corner[((int64_t)ib * g.ns + j) * ps.B + gb];
#pragma unroll
            for (int d = 16; d > 0; d >>= 1) t += __shfl_xor_sync(0xffffffffu, t, d);
            if (lane == 0) s_tr = t;
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
            issue_product(d1, smem_addr(sm.T), smem_addr(sm.OT));  // D1 = T . O_b
            mma_commit(&sm.mbar);
        }
        ok = __syncthreads_and(wait_product(&sm.mbar, parity));
        parity ^= 1u;
        if (!ok) break;
        fence_after_sync();
        // D1 (<= 128, exact in bf16: the upper half of the fp32 word) -> XA, row r = tid
        for (int cb = 0; cb < kMT / 32; ++cb) {
            uint32_t v[32];
            tmem_ld32(d1 + lanes + cb * 32, v);
            tmem_wait_ld();
#pragma unroll
            for (int q = 0; q < 4; ++q) {
                uint32_t w[4];
#pragma unroll
                for (int e = 0; e < 4; ++e) w[e] = (v[q * 8 + 2 * e] >> 16) | (v[q * 8 + 2 * e + 1] & 0xFFFF0000u);
                *reinterpret_cast<uint4 *>(sm.XA + kmaj_off(tid, cb * 32 + q * 8)) = make_uint4(w[0], w[1], w[2], w[3]);
            }
        }
        fence_async_smem();
        fence_before_sync();
        __syncthreads();
        fence_after_sync();
        if (tid == 0) {
            issue_product(d2, smem_addr(sm.XA), smem_addr(sm.T));  // D2 = D1 . T^t
            mma_commit(&sm.mbar);
        }
        ok = __syncthreads_and(wait_product(&sm.mbar, parity));
        parity ^= 1u;
        if (!ok) break;
        fence_after_sync();
        // epilogue: counts + carries into the stage, then 512-byte row stores
        const int32_t base = s_tr + sm.lp[tid];
        for (int cb = 0; cb < kMT / 32; ++cb) {
            uint32_t v[32];
            tmem_ld32(d2 + lanes + cb * 32, v);
            tmem_wait_ld();
#pragma unroll
            for (int e = 0; e < 32; e += 4) {
                const int c = cb * 32 + e;
                int4 o;
                o.x = __float2int_rz(__uint_as_float(v[e])) + base + sm.gp[c];
                o.y = __float2int_rz(__uint_as_float(v[e + 1])) + base + sm.gp[c + 1];
                o.z = __float2int_rz(__uint_as_float(v[e + 2])) + base + sm.gp[c + 2];
                o.w = __float2int_rz(__uint_as_float(v[e + 3])) + base + sm.gp[c + 3];
                *reinterpret_cast<int4 *>(&sm.out[tid][c]) = o;
            }
        }
        fence_before_sync();
        __syncthreads();
        const int c = 4 * lane;
        if (C0 + c < g.P)
            for (int rr = warp; rr < nr; rr += 4)
                *reinterpret_cast<int4 *>(ps.out + ((int64_t)gb * g.H + R0 + rr) * g.P + C0 + c) =
                    *reinterpret_cast<const int4 *>(&sm.out[rr][c]);
    }
    if (!ok) {
        if (tid == 0) atomicOr(err, 2);
        wait_product(&sm.mbar, parity ^ 1u);  // a last bounded wait for the product in flight
    }
    fence_before_sync();
    __syncthreads();
    fence_after_sync();
    if (warp == 0)
        asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(kTmemCols) : "memory");
}

}  // namespace

size_t mma_smem_bytes() { return sizeof(MmaSmem) + 1024; }

int launch_tiles_mma(const PlaneSet &ps, int *err, cudaStream_t st, const Prof *prof)
{
    // the shared-memory limit is an attribute of the kernel on the current
    // device: set it once per device, under a lock
    static std::mutex mu;
    static bool done[64] = {false};
    int dev = 0;
    cudaGetDevice(&dev);
    {
        std::lock_guard<std::mutex> lk(mu);
        if (dev >= 0 && dev < 64 && !done[dev]) {
            cudaFuncSetAttribute(k_tiles_mma, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)mma_smem_bytes());
            done[dev] = true;
        }
    }
    prof_mark(prof, KID_TILES_MMA, 0, st);
    launch_pdl(k_tiles_mma, dim3(ps.g.ns, ps.g.nb, ps.nchan), kMThreads, mma_smem_bytes(), st, ps, err);
    prof_mark(prof, KID_TILES_MMA, 1, st);
    return cudaPeekAtLastError() == cudaSuccess ? 1 : -1;
}

}  // namespace ih
