// S3 + S4 (+ S7b, S7c), mixed precision on the 5th-generation tensor cores.
//
// Forward (per 128-sample tile, 256 threads): gather the FP16 hash-table
// features of every level (Sec. 4.1, NGP; x-adjacent corners that share an
// aligned pair of entries in one 8-byte load) and interpolate them in FP32, store
// them as FP16 into shared memory, then run the density MLP and the shared
// colour MLP (Sec. 4.1) as a chain of tcgen05 MMAs, M = 128 samples, FP16
// operands in shared memory, FP32 accumulators in tensor memory.  Each
// epilogue (ReLU, FP16 cast) goes tensor memory -> registers -> shared memory
// and feeds the next MMA.  The FP16 features of the tile are also written to
// global memory (64 bytes per sample) so that the backward does not re-gather
// 512 bytes per sample from the tables.  Two forms: k_field_tc, whose threads
// gather a tile and then run its chain (1-3 CTAs per SM), and k_field_fws, whose
// eight gather warps fill one of two feature buffers while its four MMA /
// epilogue warps run the previous tile's chain (2 CTAs per SM; the default).
// k_field_fws keeps its features and each layer's output in tensor memory as
// the next layer's A operand (tcgen05.mma with A from tensor memory), so its
// shared memory holds only the weights and its operands stay out of the L1TEX
// data pipe that its table gathers need.
//
// Backward (per tile, one CTA per SM): warps 0-7 reload the features and
// either recompute the MLP activations or (a training step whose forward stored
// them) copy them back with bulk copies, then per layer two MMAs: the input gradient
// dX = delta * W (W read MN-major from the same shared buffer the forward
// reads K-major) and the weight gradient dW += delta^T * X (both operands read
// MN-major from the sample-major buffers; the output rows of dW are padded to
// M = 128 and the padding rows are never read).  The weight gradients stay in
// tensor memory for the whole persistent loop and are added to the FP32
// gradient buffer when the CTA moves to another slot and at exit.  The
// feature gradient of a tile goes through a two-buffer shared-memory ring to
// the scatter warps (4, or 8 with stored activations), which scatter-add it into
// the FP32 table gradients with fire-and-forget reductions (one thread per sample
// and level group; x-adjacent corners that
// share an aligned pair of entries in one 16-byte reduction) while warps 0-7
// run the next tile's MMA chain: the L1 reduction traffic of one tile overlaps
// the tensor-core latency chain of the next.
//
// All mbarrier waits are bounded in time; a wait that gives up sets the
// timeout status bit, stops the tile loop of the CTA, waits (bounded) for the
// tensor core and frees the tensor memory before returning.  Decisions that
// end the MMA warps' loop are made uniform over those warps (bar.red.or) and
// also release the scatter warps' waits through a shared abort flag.
//
// View-direction variant (VD): the colour MLP's input is [g | SH_16(d)], a
// [128 x 32] operand whose columns 16..31 hold the spherical harmonics of each
// sample's ray direction (hi and lo parts like every other operand).  In the
// core-matrix layout the first 16 columns of a 32-column buffer sit exactly
// where a 16-column buffer would put them, so the input-gradient MMA of that
// layer runs with N = 16 on the [64 x 32] weights and yields dg alone.
#include "kernels.cuh"
#include "tc.cuh"

namespace snk {
namespace {

constexpr int TM = 128;  // samples per tile = MMA M
constexpr int TT = 256;  // threads of the MMA / epilogue warps (warps 0-7)
// Backward: threads of the scatter warps (warps 8..), one per sample of a tile and level
// group: 4 warps (every level of a sample) when the MMA warps recompute the forward, 8 warps
// (even / odd levels) when they read stored activations -- their chain is then short
// enough that the scatter binds, and a second thread per sample shortens it.
__host__ __device__ constexpr int scatter_threads(bool sv) { return sv ? 256 : 128; }
constexpr uint32_t kChainBar = 1;  // named barrier of the 256 MMA / epilogue threads
// Backward: thread 0 issues each layer's input-gradient MMAs (the chain waits for them before the
// layer's epilogue); this thread issues the layer's weight-gradient MMAs into their own mbarrier,
// waited one layer later.  Issuing a tcgen05.mma takes tens of cycles whatever its N, so the weight
// gradients (8 of a layer's up to 16 MMAs) would otherwise lengthen every round of the chain.
constexpr int kWIssuer = 32;
// Scatter: levels up to this resolution (cells of 3.3 m and more on a 512 m tile) sum the terms of
// a warp's samples that share a cell before reducing; finer levels rarely share one (28-32
// distinct cells per 32 consecutive samples at N >= 153), where the shuffles would not pay.
constexpr int kRunMaxN = 160;
// Split FP16 operands (Markidis et al. 2018): every activation and delta x
// that feeds an MMA is carried as hi = fp16(x) and lo = fp16((x - hi) * 2^11);
// a layer runs two MMAs, hi * W and lo * W, into separate tensor-memory
// accumulators and the epilogue adds D_hi + 2^-11 D_lo.  With the FP16
// weights of the working copy exact, the layer then carries ~22 bits, so
// the cancellation in 64-term dot products does not amplify 16-bit
// rounding (the weight-gradient MMAs use the high parts only).
constexpr float kLoScale = 2048.0f, kLoInv = 1.0f / 2048.0f;

constexpr int cmax(int a, int b) { return a > b ? a : b; }

template <int IN, bool BWD, bool VD>
struct L {
  static constexpr int INP = IN < 16 ? 16 : IN;  // layer-1 K padded to the MMA K step
  static constexpr int CIN = VD ? 32 : 16;        // colour input width (K of the first colour layer)
  // backward deltas (high parts) first: the padded MN-major reads of dW run up
  // to 32 KB past a delta buffer and must stay inside the allocation
  static constexpr int DA = 0;                                 // [128 x 64]
  static constexpr int DB = BWD ? DA + TM * 64 * 2 : 0;        // [128 x 64]
  static constexpr int DG = BWD ? DB + TM * 64 * 2 : 0;        // [128 x 16]
  static constexpr int D3 = BWD ? DG + TM * 16 * 2 : 0;        // [128 x 16]
  // Low parts (x 2^11) of the forward operands, while the forward runs (in a forward or a
  // recomputing backward; the deltas' low parts are in tensor memory, A_LO; the region also keeps
  // the dW MMAs' padded reads past the delta buffers inside the allocation).
  // The forward keeps one [128 x 64] buffer for every operand (hi and lo): a layer's epilogue
  // runs only after the MMA that read the layer's input has completed, so the output can
  // overwrite it.  The backward keeps every activation for its weight-gradient MMAs.
  static constexpr int LO = BWD ? D3 + TM * 16 * 2 : 0;
  static constexpr int XL0 = LO;                               // [128 x INP] features
  static constexpr int XLA = BWD ? XL0 + TM * INP * 2 : LO;    // [128 x 64] h1, then c1
  static constexpr int XLB = BWD ? XLA + TM * 64 * 2 : LO;     // [128 x 64] h2, then g, then c2
  static constexpr int XL3 = XLB;
  static constexpr int LO_END =
      LO + (BWD ? cmax(TM * INP * 2 + 2 * TM * 64 * 2, 2 * TM * 64 * 2 + 2 * TM * 16 * 2) : TM * 64 * 2);
  // high parts of the forward operands
  static constexpr int X0 = LO_END;                            // [128 x INP]
  static constexpr int X1 = BWD ? X0 + TM * INP * 2 : X0;      // h1  [128 x 64]
  static constexpr int X2 = BWD ? X1 + TM * 64 * 2 : X0;       // h2
  static constexpr int X3 = BWD ? X2 + TM * 64 * 2 : X0;       // g [128 x CIN]
  static constexpr int X4 = BWD ? X3 + TM * CIN * 2 : X0;      // c1
  static constexpr int X5 = BWD ? X4 + TM * 64 * 2 : X0;       // c2
  static constexpr int W1 = BWD ? X5 + TM * 64 * 2 : X0 + TM * 64 * 2;  // [64 x INP]
  static constexpr int W2 = W1 + 64 * INP * 2;                 // [64 x 64]
  static constexpr int W3 = W2 + 64 * 64 * 2;                  // [16 x 64]
  static constexpr int V1 = W3 + 16 * 64 * 2;                  // [64 x CIN]
  static constexpr int V2 = V1 + 64 * CIN * 2;                 // [64 x 64]
  static constexpr int V3 = V2 + 64 * 64 * 2;                  // [16 x 64]
  static constexpr int END = V3 + 16 * 64 * 2;
  // backward: two [128 x (IN + 4)] binary32 feature-gradient buffers handed to the scatter warps
  // (rows padded by 16 B against bank conflicts)
  static constexpr int DFS = IN + 4;
  static constexpr int DF = END;
  static constexpr int DF_BYTES = BWD ? 2 * TM * DFS * 4 : 0;
  // mbarriers (MMA commit, ring full[2] / empty[2]), TMEM address, tile info[2], abort flag,
  // weight-gradient commits [2], stored activations landed [6]
  static constexpr int MISC = DF + DF_BYTES;
  static constexpr int SMEM = MISC + 192;
  static constexpr uint32_t TCOLS = BWD ? 512 : 128;
  // tensor-memory columns: 0..63 accumulator of the high parts; C_DL the low parts
  static constexpr uint32_t C_W1 = 64, C_W2 = 128, C_W3 = 192, C_V2 = 256, C_V3 = 320, C_V1 = 384;
  static constexpr uint32_t C_DL = BWD ? 448 : 64;
  // backward: the scaled low parts of a layer's delta, the A operand of the next input-gradient
  // MMA (K <= 64: 32 columns, between dW1's accumulator and dW2's)
  static constexpr uint32_t A_LO = 96;
  static_assert(!BWD || (C_W1 + INP <= A_LO && A_LO + 32 <= C_W2), "tensor-memory columns of the delta low parts");
  // Stored activations of a tile (high parts, FP16, in the layout above), written by the
  // forward of a training step and copied back by the backward instead of recomputed:
  // h1, h2 [128 x 64], then with a colour network g [128 x CIN], c1, c2 [128 x 64].
  static constexpr int A1 = 0, A2 = TM * 64 * 2, A3 = 2 * TM * 64 * 2, A4 = A3 + TM * CIN * 2, A5 = A4 + TM * 64 * 2;
  __host__ __device__ static constexpr int act_bytes(bool col) { return col ? A5 + TM * 64 * 2 : A3; }
};

// Paired binary32 arithmetic (fma / mul .rn.f32x2): two lanes of IEEE binary32, each rounded as
// the scalar instruction would round it.
__device__ __forceinline__ uint64_t f2pk(float a, float b) {
  uint64_t d;
  asm("mov.b64 %0, {%1, %2};" : "=l"(d) : "f"(a), "f"(b));
  return d;
}
__device__ __forceinline__ void f2upk(uint64_t v, float &a, float &b) { asm("mov.b64 {%0, %1}, %2;" : "=f"(a), "=f"(b) : "l"(v)); }
__device__ __forceinline__ uint64_t ffma2(uint64_t a, uint64_t b, uint64_t c) {
  uint64_t d;
  asm("fma.rn.f32x2 %0, %1, %2, %3;" : "=l"(d) : "l"(a), "l"(b), "l"(c));
  return d;
}
__device__ __forceinline__ uint64_t fmul2(uint64_t a, uint64_t b) {
  uint64_t d;
  asm("mul.rn.f32x2 %0, %1, %2;" : "=l"(d) : "l"(a), "l"(b));
  return d;
}

__device__ __forceinline__ uint32_t pack_h2(float a, float b) {
  const __half2 v = __floats2half2_rn(a, b);
  return *reinterpret_cast<const uint32_t *>(&v);
}
__device__ __forceinline__ float2 unpack_h2(uint32_t u) {
  __half2 v = *reinterpret_cast<__half2 *>(&u);
  return __half22float2(v);
}

// The MMA helpers below are issued by one thread, one tcgen05.mma per K step of 16: each builds
// its two shared-memory descriptors once and steps them by adding the K step's byte offset / 16 to
// the address field (the addresses stay below 2^18, so the 14-bit field never carries), and all
// sizes are compile-time constants, so the issuing thread spends a few instructions per MMA instead
// of rebuilding both descriptors.

// D[128 x N] = A[128 x K] * B^T, A K-major (128 rows), B = weights [N x K] K-major (N rows).
template <int K, int N>
__device__ __forceinline__ void mma_fwd(uint32_t d, uint32_t a, uint32_t b) {
  constexpr uint32_t id = tc::idesc_f16(TM, N, 0, 0);
  const uint64_t da = tc::desc(a, (TM / 8) * 128, 128), db = tc::desc(b, (N / 8) * 128, 128);
#pragma unroll
  for (int j = 0; j < K / 16; ++j)
    tc::mma_f16(d, da + (uint64_t)(j * 2 * (TM / 8) * 8), db + (uint64_t)(j * 2 * (N / 8) * 8), id, j > 0);
}

// The same with A[128 x K] in tensor memory (8 columns a K step, from a_tmem on).
template <int K, int N>
__device__ __forceinline__ void mma_fwd_ts(uint32_t d, uint32_t a_tmem, uint32_t b) {
  constexpr uint32_t id = tc::idesc_f16(TM, N, 0, 0);
  const uint64_t db = tc::desc(b, (N / 8) * 128, 128);
#pragma unroll
  for (int j = 0; j < K / 16; ++j)
    tc::mma_f16_ts(d, a_tmem + (uint32_t)(j * 8), db + (uint64_t)(j * 2 * (N / 8) * 8), id, j > 0);
}

// D[128 x N] = delta[128 x K] * W, delta K-major, W stored [K rows x N] and read MN-major.
template <int K, int N>
__device__ __forceinline__ void mma_dx(uint32_t d, uint32_t delta, uint32_t w) {
  constexpr uint32_t id = tc::idesc_f16(TM, N, 0, 1);
  const uint64_t da = tc::desc(delta, (TM / 8) * 128, 128), db = tc::desc(w, 128, (K / 8) * 128);
#pragma unroll
  for (int j = 0; j < K / 16; ++j)
    tc::mma_f16(d, da + (uint64_t)(j * 2 * (TM / 8) * 8), db + (uint64_t)(j * 16), id, j > 0);
}

// D[128 (rows = output units, padded) x N] (+)= delta^T * X over the 128 samples; both read MN-major.
template <int N>
__device__ __forceinline__ void mma_dw(uint32_t d, uint32_t delta, uint32_t x, uint32_t accumulate) {
  constexpr uint32_t id = tc::idesc_f16(TM, N, 1, 1);
  const uint64_t da = tc::desc(delta, 128, (TM / 8) * 128), db = tc::desc(x, 128, (TM / 8) * 128);
#pragma unroll
  for (int j = 0; j < TM / 16; ++j)
    tc::mma_f16(d, da + (uint64_t)(j * 16), db + (uint64_t)(j * 16), id, (j > 0) || accumulate);
}

// The same with delta in tensor memory (8 columns a K step from a_tmem).
template <int K, int N>
__device__ __forceinline__ void mma_dx_ts(uint32_t d, uint32_t a_tmem, uint32_t w) {
  constexpr uint32_t id = tc::idesc_f16(TM, N, 0, 1);
  const uint64_t db = tc::desc(w, 128, (K / 8) * 128);
#pragma unroll
  for (int j = 0; j < K / 16; ++j) tc::mma_f16_ts(d, a_tmem + (uint32_t)(j * 8), db + (uint64_t)(j * 16), id, j > 0);
}

// Copy a row-major [rows x cols] 16-bit matrix from global into the core layout (R = rpad rows,
// C = cpad columns), zero-padding, by the first nthreads threads (the MMA / epilogue threads).
__device__ __forceinline__ void load_weights(uint8_t *dst, const uint16_t *src, int rows, int cols, int rpad, int cpad,
                                             int nthreads = TT) {
  for (int e = threadIdx.x; e < rpad * cpad; e += nthreads) {
    const int r = e / cpad, c = e % cpad;
    const uint16_t v = (r < rows && c < cols) ? src[r * cols + c] : (uint16_t)0;
    *reinterpret_cast<uint16_t *>(dst + tc::core_off(r, c, rpad)) = v;
  }
}

// Epilogue of a [128 x 64] accumulator pair: this thread's row r and its 32-column half,
// v = D_hi + 2^-11 D_lo.  mode 0: v = ReLU(v); mode 1: v *= (mask > 0) (mask from a
// [128 x 64] activation buffer).  v is written as hi (out) and scaled lo (out_lo).
// LO = false: the layer had no low-part MMA (E4M3 first layer, whose input is exact in
// FP16); scale multiplies the sum (the E4M3 input's per-slot scale, else 1).
// gout (nullable): a global copy of the high parts in the same layout (stored activations),
// written with the streaming (evict-first) hint so that it does not push the hash tables out of L2.
template <int MODE, bool LO = true>
__device__ __forceinline__ void epi64(uint32_t taddr, uint32_t taddr_lo, uint8_t *out, uint8_t *out_lo,
                                      const uint8_t *mask, int r, int ch, float scale = 1.0f,
                                      uint8_t *gout = nullptr) {
  float v[32];
  {
    float a[16], b[16], c[16], d[16];
    tc::ld16(taddr + ch * 32, a);
    tc::ld16(taddr + ch * 32 + 16, b);
    if (LO) {
      tc::ld16(taddr_lo + ch * 32, c);
      tc::ld16(taddr_lo + ch * 32 + 16, d);
    }
    tc::wait_ld();
#pragma unroll
    for (int i = 0; i < 16; ++i) {
      v[i] = LO ? fmaf(c[i], kLoInv, a[i]) : a[i] * scale;
      v[16 + i] = LO ? fmaf(d[i], kLoInv, b[i]) : b[i] * scale;
    }
  }
#pragma unroll
  for (int q = 0; q < 4; ++q) {
    const int c = ch * 32 + q * 8;
    const uint32_t off = tc::core_off(r, c, TM);
    uint4 m4 = make_uint4(0, 0, 0, 0);
    if (MODE == 1) m4 = *reinterpret_cast<const uint4 *>(mask + off);
    const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
    uint32_t o[4], ol[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      float x0 = v[q * 8 + 2 * p], x1 = v[q * 8 + 2 * p + 1];
      if (MODE == 0) {
        x0 = fmaxf(x0, 0.f);
        x1 = fmaxf(x1, 0.f);
      } else {
        const float2 mk = unpack_h2(mw[p]);
        x0 = mk.x > 0.f ? x0 : 0.f;
        x1 = mk.y > 0.f ? x1 : 0.f;
      }
      o[p] = pack_h2(x0, x1);
      const float2 h = unpack_h2(o[p]);
      ol[p] = pack_h2((x0 - h.x) * kLoScale, (x1 - h.y) * kLoScale);
    }
    *reinterpret_cast<uint4 *>(out + off) = make_uint4(o[0], o[1], o[2], o[3]);
    *reinterpret_cast<uint4 *>(out_lo + off) = make_uint4(ol[0], ol[1], ol[2], ol[3]);
    if (gout) __stcs(reinterpret_cast<uint4 *>(gout + off), make_uint4(o[0], o[1], o[2], o[3]));
  }
}

// Forward epilogue into tensor memory: this thread's row and 32-column half of a [128 x 64]
// accumulator pair, v = ReLU(D_hi + 2^-11 D_lo), written as the next layer's A operand: high
// parts at a_hi, scaled low parts at a_lo (this thread's lane; 16 columns from column 16 ch),
// and, if gout is given, the high parts to global in the shared-memory core layout (stored
// activations, streaming hint).  The caller waits for the stores (tc::wait_st) before the
// hand-off to the MMA issuer.
__device__ __forceinline__ void epi64_tm(uint32_t taddr, uint32_t taddr_lo, uint32_t a_hi, uint32_t a_lo, int r, int ch,
                                         uint8_t *gout) {
  // two rounds of 16 columns: fewer values live at once than loading all 32 first
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    const int c0 = ch * 32 + hf * 16;
    float a[16], c[16];
    tc::ld16(taddr + c0, a);
    tc::ld16(taddr_lo + c0, c);
    tc::wait_ld();
    uint32_t o[8], ol[8];
    const uint64_t inv2 = f2pk(kLoInv, kLoInv), sc2 = f2pk(kLoScale, kLoScale), nsc2 = f2pk(-kLoScale, -kLoScale);
#pragma unroll
    for (int p = 0; p < 8; ++p) {
      // v = D_hi + 2^-11 D_lo, ReLU, high part h = FP16(v), scaled low part (v - h) 2^11 computed as
      // fma(-h, 2^11, v 2^11): exact, as the difference and the power-of-two scaling are
      float x0, x1;
      f2upk(ffma2(f2pk(c[2 * p], c[2 * p + 1]), inv2, f2pk(a[2 * p], a[2 * p + 1])), x0, x1);
      x0 = fmaxf(x0, 0.f);
      x1 = fmaxf(x1, 0.f);
      o[p] = pack_h2(x0, x1);
      const float2 h = unpack_h2(o[p]);
      float l0, l1;
      f2upk(ffma2(f2pk(h.x, h.y), nsc2, fmul2(f2pk(x0, x1), sc2)), l0, l1);
      ol[p] = pack_h2(l0, l1);
    }
    tc::st8(a_hi + c0 / 2, o);
    tc::st8(a_lo + c0 / 2, ol);
    if (gout) {
#pragma unroll
      for (int q = 0; q < 2; ++q)
        __stcs(reinterpret_cast<uint4 *>(gout + tc::core_off(r, c0 + q * 8, TM)),
               make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]));
    }
  }
}

// 16 floats as 8 columns of FP16 pairs in tensor memory (high parts at a_hi, scaled low parts
// at a_lo) and, if gbuf is given, the high parts to global as the [128 x 16] core-layout row r.
__device__ __forceinline__ void store16_tm(uint32_t a_hi, uint32_t a_lo, int r, const float (&v)[16],
                                           uint8_t *gbuf) {
  uint32_t o[8], ol[8];
#pragma unroll
  for (int p = 0; p < 8; ++p) {
    o[p] = pack_h2(v[2 * p], v[2 * p + 1]);
    const float2 h = unpack_h2(o[p]);
    ol[p] = pack_h2((v[2 * p] - h.x) * kLoScale, (v[2 * p + 1] - h.y) * kLoScale);
  }
  tc::st8(a_hi, o);
  tc::st8(a_lo, ol);
  if (gbuf) {
#pragma unroll
    for (int q = 0; q < 2; ++q)
      __stcs(reinterpret_cast<uint4 *>(gbuf + tc::core_off(r, q * 8, TM)),
             make_uint4(o[4 * q], o[4 * q + 1], o[4 * q + 2], o[4 * q + 3]));
  }
}

// Backward epilogue: as epi64<1> (this thread's row and column half of a [128 x 64]
// accumulator pair, v = D_hi + 2^-11 D_lo kept where the [128 x 64] activation mask is positive),
// the high parts to shared memory (out: the weight-gradient MMA and the next input-gradient MMA
// read them) and the scaled low parts to tensor memory (a_lo, this thread's lane, 16 columns from
// column 16 ch: only the next input-gradient MMA reads them).  The caller waits for the tensor-
// memory stores (tc::wait_st) before the hand-off.
__device__ __forceinline__ void epi64_bwd(uint32_t taddr, uint32_t taddr_lo, uint8_t *out, uint32_t a_lo,
                                          const uint8_t *mask, int r, int ch) {
#pragma unroll
  for (int hf = 0; hf < 2; ++hf) {
    const int c0 = ch * 32 + hf * 16;
    float a[16], c[16];
    tc::ld16(taddr + c0, a);
    tc::ld16(taddr_lo + c0, c);
    tc::wait_ld();
    uint32_t ol[8];
#pragma unroll
    for (int q = 0; q < 2; ++q) {
      const uint32_t off = tc::core_off(r, c0 + q * 8, TM);
      const uint4 m4 = *reinterpret_cast<const uint4 *>(mask + off);
      const uint32_t mw[4] = {m4.x, m4.y, m4.z, m4.w};
      uint32_t o[4];
#pragma unroll
      for (int p = 0; p < 4; ++p) {
        const float2 mk = unpack_h2(mw[p]);
        const int i = q * 8 + 2 * p;
        const float x0 = mk.x > 0.f ? fmaf(c[i], kLoInv, a[i]) : 0.f;
        const float x1 = mk.y > 0.f ? fmaf(c[i + 1], kLoInv, a[i + 1]) : 0.f;
        o[p] = pack_h2(x0, x1);
        const float2 h = unpack_h2(o[p]);
        ol[q * 4 + p] = pack_h2((x0 - h.x) * kLoScale, (x1 - h.y) * kLoScale);
      }
      *reinterpret_cast<uint4 *>(out + off) = make_uint4(o[0], o[1], o[2], o[3]);
    }
    tc::st8(a_lo + c0 / 2, ol);
  }
}

// 16 floats as one FP16 row segment of a [128 x 16] shared buffer (high parts) and their scaled
// low parts as 8 tensor-memory columns of this thread's lane at a_lo.
__device__ __forceinline__ void store16_bwd(uint8_t *buf, uint32_t a_lo, int r, const float (&v)[16]) {
  uint32_t ol[8];
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    uint32_t o[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      const int i = q * 8 + 2 * p;
      o[p] = pack_h2(v[i], v[i + 1]);
      const float2 h = unpack_h2(o[p]);
      ol[q * 4 + p] = pack_h2((v[i] - h.x) * kLoScale, (v[i + 1] - h.y) * kLoScale);
    }
    *reinterpret_cast<uint4 *>(buf + tc::core_off(r, q * 8, TM)) = make_uint4(o[0], o[1], o[2], o[3]);
  }
  tc::st8(a_lo, ol);
}

// 16 columns of an accumulator pair, combined: v = D_hi + 2^-11 D_lo.
__device__ __forceinline__ void ld16_pair(uint32_t taddr, uint32_t taddr_lo, float (&v)[16]) {
  float lo[16];
  tc::ld16(taddr, v);
  tc::ld16(taddr_lo, lo);
  tc::wait_ld();
#pragma unroll
  for (int i = 0; i < 16; ++i) v[i] = fmaf(lo[i], kLoInv, v[i]);
}

// Store 16 floats as one FP16 row segment of a [128 x 16] buffer (and, if buf_lo is
// given, their scaled low parts; if gbuf is given, a global copy of the high parts).
__device__ __forceinline__ void store16(uint8_t *buf, uint8_t *buf_lo, int r, const float (&v)[16],
                                        uint8_t *gbuf = nullptr) {
#pragma unroll
  for (int q = 0; q < 2; ++q) {
    uint32_t o[4], ol[4];
#pragma unroll
    for (int p = 0; p < 4; ++p) {
      o[p] = pack_h2(v[q * 8 + 2 * p], v[q * 8 + 2 * p + 1]);
      const float2 h = unpack_h2(o[p]);
      ol[p] = pack_h2((v[q * 8 + 2 * p] - h.x) * kLoScale, (v[q * 8 + 2 * p + 1] - h.y) * kLoScale);
    }
    *reinterpret_cast<uint4 *>(buf + tc::core_off(r, q * 8, TM)) = make_uint4(o[0], o[1], o[2], o[3]);
    if (buf_lo) *reinterpret_cast<uint4 *>(buf_lo + tc::core_off(r, q * 8, TM)) = make_uint4(ol[0], ol[1], ol[2], ol[3]);
    if (gbuf) __stcs(reinterpret_cast<uint4 *>(gbuf + tc::core_off(r, q * 8, TM)), make_uint4(o[0], o[1], o[2], o[3]));
  }
}

__device__ __forceinline__ float sigm(float x) { return 1.0f / (1.0f + __expf(-x)); }

// A tile handed from the MMA warps to the scatter warps.
struct TileInfo {
  int64_t ts;       // first slot-major sample of the tile
  int32_t slot;
  int32_t n_valid;  // rows 0 .. n_valid-1 are samples of the slot
};

// SV (backward): the forward stored the tile's activations (a.acts); they are copied back
// with bulk copies instead of recomputed.
template <int IN, int G, bool COL, bool BWD, bool Q8, int KL, bool VD, int MINB, bool SV>
__global__ void __launch_bounds__(BWD ? TT + scatter_threads(SV) : TT, MINB) k_field_tc(const FieldArgs a) {
  using Y = L<IN, BWD, VD>;
  constexpr int INP = Y::INP;
  constexpr int CIN = Y::CIN;
  constexpr int ACT = Y::act_bytes(COL);
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + Y::MISC);
  uint64_t *full = mbar + 1;   // [2] the MMA warps filled DF[b] (TT arrivals)
  constexpr int TS = scatter_threads(SV);
  uint64_t *empty = mbar + 3;  // [2] the scatter warps drained DF[b] (TS arrivals)
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + Y::MISC + 40);
  TileInfo *info = reinterpret_cast<TileInfo *>(sm + Y::MISC + 48);  // [2]
  volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + Y::MISC + 80);
  // stored activations landed, one barrier a buffer, numbered in the order the backward reads
  // them: c2, c1, g (with a colour network), h2, h1, the features
  uint64_t *abar = reinterpret_cast<uint64_t *>(sm + Y::MISC + 128);  // [6]
  constexpr int kGX2 = COL ? 3 : 0, kGX1 = kGX2 + 1, kGX0 = kGX2 + 2;
  // weight-gradient MMAs completed: commit i (counted over the kernel) arrives on wbar[i & 1], so
  // neither barrier runs more than one phase ahead of the threads that wait for it
  uint64_t *wbar = reinterpret_cast<uint64_t *>(sm + Y::MISC + 96);  // [2]
  float *dfbuf = reinterpret_cast<float *>(sm + Y::DF);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int r = 32 * (warp & 3) + lane;  // TMEM lane = tile row of this thread
  const int ch = warp >> 2;             // column half
  const snk_state *st = a.state;
  snk_state *st_rw = const_cast<snk_state *>(a.state);
  const ModelDev &m = a.m;
  const GridParams &gp = m.grid;
  const uint32_t s0 = tc::smem_u32(sm);

  if (t == 0) {
    tc::mbar_init(mbar, 1);
    if (BWD) {
      for (int b = 0; b < 2; ++b) {
        tc::mbar_init(full + b, TT);
        tc::mbar_init(empty + b, TS);
      }
    }
    *abort_flag = 0;
    if (SV)
      for (int i = 0; i <= kGX0; ++i) tc::mbar_init(abar + i, 1);
    if (BWD) {
      tc::mbar_init(wbar, 1);
      tc::mbar_init(wbar + 1, 1);
    }
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, Y::TCOLS);
  // zero every operand buffer once (padding columns are never written again)
  for (int i = t; i < Y::END / 16; i += blockDim.x) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
  uint32_t phase = 0, aphase = 0;
  // weight-gradient commits issued and waited for (every MMA / epilogue thread counts them alike)
  uint32_t w_issued = 0, w_waited = 0;
  bool abort = false;
  uint32_t a_pend = 0;  // thread 0: stored-activation copies issued and not yet waited for

  int64_t r0 = 0, r1 = st->slot_base[kMaxSlots];
  if (a.slot_only >= 0) {
    r0 = st->slot_base[a.slot_only];
    r1 = r0 + st->slot_count[a.slot_only];
  }
  if (r1 > a.S) r1 = a.S;
  const int64_t n_tiles = r1 > r0 ? (r1 - r0 + TM - 1) / TM : 0;
  int cur_slot = -1;
  bool fresh = true;  // next dW MMAs start the accumulators

  // MMA / epilogue threads: wait for the MMAs committed last; uniform result over those threads
  auto sync_mma = [&]() -> bool {
    const bool ok = tc::mbar_wait(mbar, phase);
    if (ok) phase ^= 1u;
    tc::fence_after_sync();
    return !tc::bar_or(kChainBar, TT, !ok);
  };
  // backward layer: wait for this layer's input-gradient MMAs and, with wait_w, for the previous
  // layer's weight-gradient MMAs (whose operands the next epilogues may overwrite); uniform result
  auto wait_w_next = [&]() -> bool {  // the oldest weight-gradient commit not yet waited for
    const bool ok = tc::mbar_wait(wbar + (w_waited & 1u), (w_waited >> 1) & 1u);
    if (ok) ++w_waited;
    return ok;
  };
  auto sync_mma_w = [&](bool wait_w, bool pre_ok) -> bool {
    ++w_issued;  // this layer's weight-gradient commit
    bool ok = tc::mbar_wait(mbar, phase) && pre_ok;
    if (ok) phase ^= 1u;
    if (wait_w) ok = wait_w_next() && ok;
    tc::fence_after_sync();
    return !tc::bar_or(kChainBar, TT, !ok);
  };
  // stored activations: every MMA / epilogue thread waits for buffer gi's copy before the
  // weight-gradient MMAs and the masks read it (false: the bounded wait gave up)
  auto wait_act = [&](int gi) -> bool {
    if (!SV) return true;
    const bool ok = tc::mbar_wait(abar + gi, aphase);
    if (ok && t == 0) a_pend &= ~(1u << gi);
    return ok;
  };
  // after an epilogue: make smem writes visible to the tensor core and TMEM reads ordered
  auto handoff = [&]() {
    tc::wait_st();  // the backward's delta low parts in tensor memory
    tc::fence_async_smem();
    tc::fence_before_sync();
    tc::bar_sync(kChainBar, TT);
    tc::fence_after_sync();
  };

  // add the dW accumulators of slot k to the FP32 gradients (BWD only)
  auto flush = [&](int k) {
    if (!BWD) return;
    float *gs = a.grads + (int64_t)k * m.tile_params;
    float *gc = a.grads + m.colour_base + (m.shared_colour ? 0 : (int64_t)k * m.colour_params);
    struct R {
      uint32_t col;
      int ncol, out, in;
      float *dst;
    };
    const R regs[6] = {{Y::C_W1, INP, 64, IN, gs + m.w1}, {Y::C_W2, 64, 64, 64, gs + m.w2},
                       {Y::C_W3, 64, G, 64, gs + m.w3},   {Y::C_V1, CIN, 64, VD ? CIN : G, gc + m.v1},
                       {Y::C_V2, 64, 64, 64, gc + m.v2},  {Y::C_V3, 64, 3, 64, gc + m.v3}};
    const int nreg = COL ? 6 : 3;
    // E4M3 first layer: the dW1 MMAs read the codes' values; the layer's input is scale x value
    const float s1 = Q8 ? e4m3_scale(a.amax[k]) : 1.0f;
    for (int q = 0; q < nreg; ++q) {
      const R &g = regs[q];
      if ((warp & 3) >= 2) continue;  // rows >= 64 are padding
      const float sc = q == 0 ? s1 : 1.0f;
      for (int c0 = ch * 16; c0 < g.ncol; c0 += 32) {
        float v[16];
        tc::ld16(trow + g.col + c0, v);
        tc::wait_ld();
        if (r < g.out) {
#pragma unroll
          for (int i = 0; i < 16; ++i)
            if (c0 + i < g.in && v[i] != 0.f) atomicAdd(g.dst + (int64_t)r * g.in + c0 + i, v[i] * sc);
        }
      }
    }
    fresh = true;
  };

  if (BWD && t >= TT) {
    // ---- scatter warps: add each tile's feature gradient, weighted by the trilinear
    // weights, into the FP32 table gradients (float2 reductions, one thread per sample and
    // level group); they run while the MMA warps work on the next tile ----
    const int s = (t - TT) % TM, lq = (t - TT) / TM;  // sample of the tile, level group
    const int lane = t & 31;                           // a warp: 32 consecutive samples, one level group
    const uint64_t keep = l2_keep();                   // the gradients stay in L2
    int j = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      if (slot_of(st, r0 + tile * TM) < 0) continue;  // the MMA warps skip the same tiles
      const int b = j & 1;
      const int w = tc::mbar_wait_or_abort(full + b, (j >> 1) & 1, abort_flag);
      if (w == 2) {
        atomicOr(&st_rw->status, kStatusTimeout);
        *abort_flag = 1;
      }
      if (__any_sync(0xffffffffu, w != 0)) break;  // uniform over the warp: its lanes shuffle below
      const TileInfo ti = info[b];
      const bool sv = s < ti.n_valid;
      const int64_t idx = ti.ts + s;
      float xyz[3] = {0.f, 0.f, 0.f};
      if (sv) {
#pragma unroll
        for (int q = 0; q < 3; ++q) xyz[q] = a.xyz[idx * 3 + q];
      }
      const float *dfr = dfbuf + (b * TM + s) * Y::DFS;
      float2 *gt0 = reinterpret_cast<float2 *>(a.grads + (int64_t)ti.slot * m.tile_params);
      for (int l = lq; l < gp.L; l += TS / TM) {
        const int N = gp.res[l];
        const bool dense = gp.dense[l] != 0;
        int ci[3];
        float fr[3];
#pragma unroll
        for (int q = 0; q < 3; ++q) grid_cell(xyz[q], N, ci[q], fr[q]);
        const float2 d = sv ? *reinterpret_cast<const float2 *>(dfr + 2 * l) : make_float2(0.f, 0.f);
        if (dense && a.cell_grad) {
          // dense level: the warp's samples that share a cell (consecutive samples along a ray)
          // sum their 8 corner terms first; the run's last lane adds them to the cell's 64-byte
          // block of the cell-major accumulator in four 16-byte reductions
          const uint32_t key = sv ? (uint32_t)ci[0] + (uint32_t)N * ((uint32_t)ci[1] + (uint32_t)N * (uint32_t)ci[2])
                                  : 0xffffffffu;
          float v[16];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float wc = ((c & 1) ? fr[0] : 1.0f - fr[0]) * ((c & 2) ? fr[1] : 1.0f - fr[1]) *
                             ((c & 4) ? fr[2] : 1.0f - fr[2]);
            v[2 * c] = wc * d.x;
            v[2 * c + 1] = wc * d.y;
          }
          if (run_sums(v, key, lane) && sv) {
            float *q = a.cell_grad + ((int64_t)ti.slot * gp.n_cells + gp.cell_off[l] + key) * 16;
#pragma unroll
            for (int k = 0; k < 16; k += 4) red_keep_v4(q + k, v[k], v[k + 1], v[k + 2], v[k + 3], keep);
          }
        } else if (N <= kRunMaxN) {
          // coarse hashed level (cells of a few metres): the same run sums, then the run's last
          // lane adds the 8 corner sums through the hash, x-adjacent pairs merged as below
          const uint32_t key = sv ? (uint32_t)ci[0] + (uint32_t)N * ((uint32_t)ci[1] + (uint32_t)N * (uint32_t)ci[2])
                                  : 0xffffffffu;
          float v[16];
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const float wc = ((c & 1) ? fr[0] : 1.0f - fr[0]) * ((c & 2) ? fr[1] : 1.0f - fr[1]) *
                             ((c & 4) ? fr[2] : 1.0f - fr[2]);
            v[2 * c] = wc * d.x;
            v[2 * c + 1] = wc * d.y;
          }
          if (run_sums(v, key, lane) && sv) {
            float2 *gt = gt0 + gp.offset[l];
#pragma unroll
            for (int c = 0; c < 8; c += 2) {
              const uint32_t e0 = grid_index(ci[0], ci[1] + ((c >> 1) & 1), ci[2] + ((c >> 2) & 1), N, dense,
                                             (uint32_t)gp.T - 1u);
              const uint32_t e1 = grid_index(ci[0] + 1, ci[1] + ((c >> 1) & 1), ci[2] + ((c >> 2) & 1), N, dense,
                                             (uint32_t)gp.T - 1u);
              red_pair_sums(gt, e0, e1, make_float2(v[2 * c], v[2 * c + 1]), make_float2(v[2 * c + 2], v[2 * c + 3]),
                            keep);
            }
          }
        } else if (sv) {
          float2 *gt = gt0 + gp.offset[l];
          // corners c and c + 1 differ in x only; red_pair merges them when they share an aligned pair
#pragma unroll
          for (int c = 0; c < 8; c += 2) {
            const uint32_t e0 = grid_index(ci[0], ci[1] + ((c >> 1) & 1), ci[2] + ((c >> 2) & 1), N, dense,
                                           (uint32_t)gp.T - 1u);
            const uint32_t e1 = grid_index(ci[0] + 1, ci[1] + ((c >> 1) & 1), ci[2] + ((c >> 2) & 1), N, dense,
                                           (uint32_t)gp.T - 1u);
            const float wyz = ((c & 2) ? fr[1] : 1.0f - fr[1]) * ((c & 4) ? fr[2] : 1.0f - fr[2]);
            red_pair(gt, e0, e1, (1.0f - fr[0]) * wyz, fr[0] * wyz, d, keep);
          }
        }
      }
      tc::mbar_arrive(empty + b);
      ++j;
    }
  } else {
  int jt = 0;  // tiles handed to the scatter warps
  for (int64_t tile = blockIdx.x; tile < n_tiles && !abort; tile += gridDim.x) {
    const int64_t ts = r0 + tile * TM;
    const int slot = slot_of(st, ts);
    if (slot < 0) continue;
    if (slot != cur_slot) {
      if (cur_slot >= 0) flush(cur_slot);
      tc::bar_sync(kChainBar, TT);
      const uint16_t *P = a.params_lp + (int64_t)slot * m.tile_params;
      const uint16_t *C = a.params_lp + m.colour_base + (m.shared_colour ? 0 : (int64_t)slot * m.colour_params);
      load_weights(sm + Y::W1, P + m.w1, 64, IN, 64, INP);
      load_weights(sm + Y::W2, P + m.w2, 64, 64, 64, 64);
      load_weights(sm + Y::W3, P + m.w3, G, 64, 16, 64);
      if (COL) {
        load_weights(sm + Y::V1, C + m.v1, 64, VD ? CIN : G, 64, CIN);
        load_weights(sm + Y::V2, C + m.v2, 64, 64, 64, 64);
        load_weights(sm + Y::V3, C + m.v3, 3, 64, 16, 64);
      }
      cur_slot = slot;
      handoff();
    }
    const int64_t slot_end = (int64_t)st->slot_base[slot] + st->slot_count[slot];
    const int64_t idx = ts + r;
    const bool valid = idx < slot_end && idx < r1;
    // backward: this row's upstream gradient and (with stored activations) forward outputs, loaded
    // now so that their latency passes while the tile's operands arrive
    float4 up = make_float4(0.f, 0.f, 0.f, 0.f), fo = make_float4(0.f, 0.f, 0.f, 0.f);
    if (BWD && ch == 0 && valid) {
      up = reinterpret_cast<const float4 *>(a.dsr)[idx];
      if (SV) fo = reinterpret_cast<const float4 *>(a.sigma_rgb)[idx];
    }
    uint16_t *ftile = a.feat_lp + (ts / TM) * (int64_t)(2 * TM * INP);  // [hi | lo] of the tile
    // this tile's stored activations: written by a training forward, read back by the backward
    uint8_t *gact = a.acts ? reinterpret_cast<uint8_t *>(a.acts) + (ts / TM) * (int64_t)ACT : nullptr;
    if (SV && t == 0) {
      // the buffers' last readers (MMAs, mask loads) finished before the barrier that ended the
      // previous tile
      tc::fence_async_smem();
      // read once: evict first, so that the stream leaves the slot's gradient table in L2
      const uint64_t pol = tc::l2_evict_first();
      // in the order of use, each buffer on its own barrier: a layer waits only for its input
      auto copy = [&](int gi, uint8_t *dst, const void *src, uint32_t bytes) {
        tc::mbar_arrive_expect_tx(abar + gi, bytes);
        tc::bulk_g2s(dst, src, bytes, abar + gi, pol);
        a_pend |= 1u << gi;
      };
      if (COL) {
        copy(0, sm + Y::X5, gact + Y::A5, TM * 64 * 2);
        copy(1, sm + Y::X4, gact + Y::A4, TM * 64 * 2);
        copy(2, sm + Y::X3, gact + Y::A3, TM * CIN * 2);
      }
      copy(kGX2, sm + Y::X2, gact + Y::A2, TM * 64 * 2);
      copy(kGX1, sm + Y::X1, gact + Y::A1, TM * 64 * 2);
      if (!Q8) copy(kGX0, sm + Y::X0, ftile, TM * INP * 2);
    }

    // ---- features ----
    const float s1 = Q8 ? e4m3_scale(a.amax[slot]) : 1.0f;  // E4M3 first layer: the slot's scale
    if (Q8) {
      // forward: quantise the binary32 features of the gather pass and keep the codes for the
      // backward; backward: reload the codes.  Both widen them to FP16 (exact) into X0.
      const int s = t & (TM - 1), half = t >> 7;
      const int64_t sidx = ts + s;
      const bool sval = sidx < slot_end && sidx < r1;
      if (16 * half < INP) {
        uint8_t *cp = a.codes + sidx * INP + 16 * half;  // this thread's 16 codes
        uint32_t cw[4];
        if (!BWD) {
          float f[16];
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            float4 v = make_float4(0.f, 0.f, 0.f, 0.f);
            if (sval && 16 * half + 4 * j < IN)
              v = *reinterpret_cast<const float4 *>(a.feat32 + sidx * IN + 16 * half + 4 * j);
            f[4 * j] = v.x;
            f[4 * j + 1] = v.y;
            f[4 * j + 2] = v.z;
            f[4 * j + 3] = v.w;
          }
#pragma unroll
          for (int j = 0; j < 4; ++j) {
            const uint16_t c01 = e4m3x2_from_f32(fdiv(f[4 * j], s1), fdiv(f[4 * j + 1], s1));
            const uint16_t c23 = e4m3x2_from_f32(fdiv(f[4 * j + 2], s1), fdiv(f[4 * j + 3], s1));
            cw[j] = (uint32_t)c01 | ((uint32_t)c23 << 16);
          }
          *reinterpret_cast<uint4 *>(cp) = make_uint4(cw[0], cw[1], cw[2], cw[3]);
        } else {
          const uint4 v = *reinterpret_cast<const uint4 *>(cp);
          cw[0] = v.x;
          cw[1] = v.y;
          cw[2] = v.z;
          cw[3] = v.w;
        }
#pragma unroll
        for (int q = 0; q < 2; ++q) {
          uint32_t h[4];
#pragma unroll
          for (int p = 0; p < 4; ++p) {
            const uint32_t w = cw[2 * q + (p >> 1)];
            h[p] = f16x2_from_e4m3x2((uint16_t)((p & 1) ? (w >> 16) : (w & 0xffffu)));
          }
          *reinterpret_cast<uint4 *>(sm + Y::X0 + tc::core_off(s, 16 * half + 8 * q, TM)) =
              make_uint4(h[0], h[1], h[2], h[3]);
        }
      }
    } else if (!BWD) {
      const int s = t & (TM - 1), half = t >> 7;
      const uint64_t keep = l2_keep();  // the tables stay in L2
      const int64_t sidx = ts + s;
      const bool sval = sidx < slot_end && sidx < r1;
      float xyz[3] = {0.f, 0.f, 0.f};
      if (sval) {
#pragma unroll
        for (int q = 0; q < 3; ++q) xyz[q] = a.xyz[sidx * 3 + q];
      }
      const __half2 *tab0 = reinterpret_cast<const __half2 *>(a.params_lp + (int64_t)slot * m.tile_params);
      // KL levels per round: their corner loads are all issued before any is used
      for (int l0 = half; l0 < gp.L; l0 += 2 * KL) {
        __half2 hv[KL][8];
        float fr[KL][3];
#pragma unroll
        for (int k = 0; k < KL; ++k) {
          const int l = l0 + 2 * k;
#pragma unroll
          for (int c = 0; c < 8; ++c) hv[k][c] = __float2half2_rn(0.f);
          fr[k][0] = fr[k][1] = fr[k][2] = 0.f;
          if (l < gp.L && sval) {
            if (a.cells_lp && gp.dense[l])  // one 32-byte load from the cell-major copy
              gather_cell(a.cells_lp + ((int64_t)slot * gp.n_cells + gp.cell_off[l]) * 16, xyz, gp.res[l], hv[k], fr[k], keep);
            else
              gather_corners(tab0 + gp.offset[l], xyz, gp.res[l], gp.dense[l] != 0, (uint32_t)gp.T - 1u, hv[k], fr[k],
                             keep);
          }
        }
#pragma unroll
        for (int k = 0; k < KL; ++k) {
          const int l = l0 + 2 * k;
          if (l >= gp.L) break;
          const float2 f = interp_corners(hv[k], fr[k]);
          const float f0 = f.x, f1 = f.y;
          const uint32_t hp = pack_h2(f0, f1);
          const float2 hh = unpack_h2(hp);
          *reinterpret_cast<uint32_t *>(sm + Y::X0 + tc::core_off(s, 2 * l, TM)) = hp;
          *reinterpret_cast<uint32_t *>(sm + Y::XL0 + tc::core_off(s, 2 * l, TM)) =
              pack_h2((f0 - hh.x) * kLoScale, (f1 - hh.y) * kLoScale);
        }
      }
      if (IN < INP && half == 0) {
        // padding columns of the first layer's K: the shared operand buffer held the last
        // tile's activations there
#pragma unroll
        for (int c = IN; c < INP; c += 2) {
          *reinterpret_cast<uint32_t *>(sm + Y::X0 + tc::core_off(s, c, TM)) = 0u;
          *reinterpret_cast<uint32_t *>(sm + Y::XL0 + tc::core_off(s, c, TM)) = 0u;
        }
      }
      tc::bar_sync(kChainBar, TT);
      // the tile's features in the shared-memory layout, for the backward: the high parts, and
      // the low parts unless the activations are stored (the backward then needs the high parts
      // only, for dW1)
      for (int i = t; i < TM * INP * 2 / 16; i += TT) {
        __stcs(reinterpret_cast<uint4 *>(ftile) + i, reinterpret_cast<const uint4 *>(sm + Y::X0)[i]);
        if (!gact) __stcs(reinterpret_cast<uint4 *>(ftile + TM * INP) + i, reinterpret_cast<const uint4 *>(sm + Y::XL0)[i]);
      }
    } else if (!SV) {
      for (int i = t; i < TM * INP * 2 / 16; i += TT) {
        reinterpret_cast<uint4 *>(sm + Y::X0)[i] = reinterpret_cast<const uint4 *>(ftile)[i];
        reinterpret_cast<uint4 *>(sm + Y::XL0)[i] = reinterpret_cast<const uint4 *>(ftile + TM * INP)[i];
      }
    }
    handoff();
    float g[16];
    float rgb[3] = {0.f, 0.f, 0.f};
    float e0 = 0.f;  // exp(clamp(g_0, -15, 15)): the truncated-exponential gradient factor of sigma
    if constexpr (SV) {
      // sigma and rgb come from the forward's output (the stored activations are waited for
      // layer by layer below)
      if (ch == 0) {
        e0 = fminf(fmaxf(fo.x, __expf(-15.f)), __expf(15.f));
        rgb[0] = fo.y;
        rgb[1] = fo.z;
        rgb[2] = fo.w;
      }
    } else {

    // ---- forward MLP ----
    if (t == 0) {
      mma_fwd<INP, 64>(tmem, s0 + Y::X0, s0 + Y::W1);
      if (!Q8) mma_fwd<INP, 64>(tmem + Y::C_DL, s0 + Y::XL0, s0 + Y::W1);
      tc::commit(mbar);
    }
    abort = !sync_mma();
    if (abort) break;
    if (Q8)
      epi64<0, false>(trow, trow + Y::C_DL, sm + Y::X1, sm + Y::XLA, nullptr, r, ch, s1, gact ? gact + Y::A1 : nullptr);
    else
      epi64<0>(trow, trow + Y::C_DL, sm + Y::X1, sm + Y::XLA, nullptr, r, ch, 1.0f, gact ? gact + Y::A1 : nullptr);
    handoff();
    if (t == 0) {
      mma_fwd<64, 64>(tmem, s0 + Y::X1, s0 + Y::W2);
      mma_fwd<64, 64>(tmem + Y::C_DL, s0 + Y::XLA, s0 + Y::W2);
      tc::commit(mbar);
    }
    abort = !sync_mma();
    if (abort) break;
    epi64<0>(trow, trow + Y::C_DL, sm + Y::X2, sm + Y::XLB, nullptr, r, ch, 1.0f, gact ? gact + Y::A2 : nullptr);
    handoff();
    if (t == 0) {
      mma_fwd<64, 16>(tmem, s0 + Y::X2, s0 + Y::W3);
      mma_fwd<64, 16>(tmem + Y::C_DL, s0 + Y::XLB, s0 + Y::W3);
      tc::commit(mbar);
    }
    abort = !sync_mma();
    if (abort) break;
    if (ch == 0) {
      ld16_pair(trow, trow + Y::C_DL, g);
      store16(sm + Y::X3, sm + Y::XL3, r, g, (COL && gact) ? gact + Y::A3 : nullptr);
      if (!COL) {
#pragma unroll
        for (int k = 0; k < 3; ++k) rgb[k] = sigm(g[1 + k]);
      }
    } else if (VD) {
      // colour input columns 16..31: SH of the sample's ray direction
      float dir[3] = {0.f, 0.f, 1.f}, y[16];
      if (valid) {
        const uint32_t ray = a.smp_ray[idx];
#pragma unroll
        for (int q = 0; q < 3; ++q) dir[q] = a.ray_od[(int64_t)(3 + q) * a.n_rays + ray];
      }
      sh16(dir[0], dir[1], dir[2], y);
      store16(sm + Y::X3 + TM * 16 * 2, sm + Y::XL3 + TM * 16 * 2, r, y, gact ? gact + Y::A3 + TM * 16 * 2 : nullptr);
    }
    handoff();
    if (COL) {
      if (t == 0) {
        mma_fwd<CIN, 64>(tmem, s0 + Y::X3, s0 + Y::V1);
        mma_fwd<CIN, 64>(tmem + Y::C_DL, s0 + Y::XL3, s0 + Y::V1);
        tc::commit(mbar);
      }
      abort = !sync_mma();
      if (abort) break;
      epi64<0>(trow, trow + Y::C_DL, sm + Y::X4, sm + Y::XLA, nullptr, r, ch, 1.0f, gact ? gact + Y::A4 : nullptr);
      handoff();
      if (t == 0) {
        mma_fwd<64, 64>(tmem, s0 + Y::X4, s0 + Y::V2);
        mma_fwd<64, 64>(tmem + Y::C_DL, s0 + Y::XLA, s0 + Y::V2);
        tc::commit(mbar);
      }
      abort = !sync_mma();
      if (abort) break;
      epi64<0>(trow, trow + Y::C_DL, sm + Y::X5, sm + Y::XLB, nullptr, r, ch, 1.0f, gact ? gact + Y::A5 : nullptr);
      handoff();
      if (t == 0) {
        mma_fwd<64, 16>(tmem, s0 + Y::X5, s0 + Y::V3);
        mma_fwd<64, 16>(tmem + Y::C_DL, s0 + Y::XLB, s0 + Y::V3);
        tc::commit(mbar);
      }
      abort = !sync_mma();
      if (abort) break;
      if (ch == 0) {
        float o[16];
        ld16_pair(trow, trow + Y::C_DL, o);
#pragma unroll
        for (int k = 0; k < 3; ++k) rgb[k] = sigm(o[k]);
      }
      tc::fence_before_sync();
      tc::bar_sync(kChainBar, TT);
      tc::fence_after_sync();
    }
    if (ch == 0) e0 = __expf(fminf(fmaxf(g[0], -15.f), 15.f));
    }  // forward MLP (recomputed in a backward without stored activations)

    if constexpr (!BWD) {
      if (ch == 0 && valid)
        reinterpret_cast<float4 *>(a.sigma_rgb)[idx] = make_float4(__expf(g[0]), rgb[0], rgb[1], rgb[2]);
      continue;
    }

    // ---- backward ----
    // output deltas (the upstream gradient already carries the loss scale)
    if (ch == 0) {
      const float4 d = up;
      const float dg0 = d.x * e0;
      const float d3[3] = {d.y * rgb[0] * (1.f - rgb[0]), d.z * rgb[1] * (1.f - rgb[1]), d.w * rgb[2] * (1.f - rgb[2])};
      float row[16];
#pragma unroll
      for (int i = 0; i < 16; ++i) row[i] = 0.f;
      if (COL) {
#pragma unroll
        for (int k = 0; k < 3; ++k) row[k] = d3[k];
        store16_bwd(sm + Y::D3, trow + Y::A_LO, r, row);
        g[0] = dg0;  // keep dsigma's contribution to dg_0 for later
      } else {
        row[0] = dg0;
#pragma unroll
        for (int k = 0; k < 3; ++k) row[1 + k] = d3[k];
        store16_bwd(sm + Y::DG, trow + Y::A_LO, r, row);
      }
    }
    handoff();
    const uint32_t acc = fresh ? 0u : 1u;
    if (COL) {
      // dc2 = delta3 * V3, dV3 += delta3^T c2
      if (t == 0) {
        mma_dx<16, 64>(tmem, s0 + Y::D3, s0 + Y::V3);
        mma_dx_ts<16, 64>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::V3);
        tc::commit(mbar);
      }
      const bool c2_ok = wait_act(0);
      if (t == kWIssuer) {  // the weight gradient: off the chain's critical path (commit index w_issued)
        mma_dw<64>(tmem + Y::C_V3, s0 + Y::D3, s0 + Y::X5, acc);
        tc::commit(wbar + (w_issued & 1u));
      }
      abort = !sync_mma_w(false, c2_ok);
      if (abort) break;
      epi64_bwd(trow, trow + Y::C_DL, sm + Y::DA, trow + Y::A_LO, sm + Y::X5, r, ch);
      handoff();
      // dc1 = delta_c2 * V2, dV2 += delta_c2^T c1
      if (t == 0) {
        mma_dx<64, 64>(tmem, s0 + Y::DA, s0 + Y::V2);
        mma_dx_ts<64, 64>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::V2);
        tc::commit(mbar);
      }
      const bool c1_ok = wait_act(1);
      if (t == kWIssuer) {  // the weight gradient: off the chain's critical path (commit index w_issued)
        mma_dw<64>(tmem + Y::C_V2, s0 + Y::DA, s0 + Y::X4, acc);
        tc::commit(wbar + (w_issued & 1u));
      }
      abort = !sync_mma_w(true, c1_ok);
      if (abort) break;
      epi64_bwd(trow, trow + Y::C_DL, sm + Y::DB, trow + Y::A_LO, sm + Y::X4, r, ch);
      handoff();
      // dg = delta_c1 * V1 (+ dsigma term; N = 16: the g columns of V1), dV1 += delta_c1^T [g | SH]
      if (t == 0) {
        mma_dx<64, 16>(tmem, s0 + Y::DB, s0 + Y::V1);
        mma_dx_ts<64, 16>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::V1);
        tc::commit(mbar);
      }
      const bool g_ok = wait_act(2);
      if (t == kWIssuer) {  // the weight gradient: off the chain's critical path (commit index w_issued)
        mma_dw<CIN>(tmem + Y::C_V1, s0 + Y::DB, s0 + Y::X3, acc);
        tc::commit(wbar + (w_issued & 1u));
      }
      abort = !sync_mma_w(true, g_ok);
      if (abort) break;
      if (ch == 0) {
        float dg[16];
        float dgl[16];
        tc::ld16(trow, dg);
        tc::ld16(trow + Y::C_DL, dgl);
        tc::wait_ld();
#pragma unroll
        for (int i = 0; i < 16; ++i) dg[i] = fmaf(dgl[i], kLoInv, dg[i]);
        dg[0] += g[0];
        store16_bwd(sm + Y::DG, trow + Y::A_LO, r, dg);
      }
      handoff();
    }
    // dh2 = delta_g * W3 (masked by h2), dW3 += delta_g^T h2 (the first layer without a colour net)
    if (t == 0) {
      mma_dx<16, 64>(tmem, s0 + Y::DG, s0 + Y::W3);
      mma_dx_ts<16, 64>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::W3);
      tc::commit(mbar);
    }
    const bool h2_ok = wait_act(kGX2);
    if (t == kWIssuer) {  // the weight gradient: off the chain's critical path (commit index w_issued)
      mma_dw<64>(tmem + Y::C_W3, s0 + Y::DG, s0 + Y::X2, acc);
      tc::commit(wbar + (w_issued & 1u));
    }
    abort = !sync_mma_w(COL, h2_ok);
    if (abort) break;
    epi64_bwd(trow, trow + Y::C_DL, sm + Y::DA, trow + Y::A_LO, sm + Y::X2, r, ch);
    handoff();
    // dh1 = delta_h2 * W2 (masked by h1), dW2 += delta_h2^T h1
    if (t == 0) {
      mma_dx<64, 64>(tmem, s0 + Y::DA, s0 + Y::W2);
      mma_dx_ts<64, 64>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::W2);
      tc::commit(mbar);
    }
    const bool h1_ok = wait_act(kGX1);
    if (t == kWIssuer) {  // the weight gradient: off the chain's critical path (commit index w_issued)
      mma_dw<64>(tmem + Y::C_W2, s0 + Y::DA, s0 + Y::X1, acc);
      tc::commit(wbar + (w_issued & 1u));
    }
    abort = !sync_mma_w(true, h1_ok);
    if (abort) break;
    epi64_bwd(trow, trow + Y::C_DL, sm + Y::DB, trow + Y::A_LO, sm + Y::X1, r, ch);
    handoff();
    // dfeat = delta_h1 * W1, dW1 += delta_h1^T feat
    if (t == 0) {
      mma_dx<64, INP>(tmem, s0 + Y::DB, s0 + Y::W1);
      mma_dx_ts<64, INP>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::W1);
      tc::commit(mbar);
    }
    const bool f_ok = Q8 || wait_act(kGX0);  // E4M3: the first layer's codes are reloaded, not copied
    if (t == kWIssuer) {  // the weight gradient: off the chain's critical path (commit index w_issued)
      mma_dw<INP>(tmem + Y::C_W1, s0 + Y::DB, s0 + Y::X0, acc);
      tc::commit(wbar + (w_issued & 1u));
    }
    abort = !sync_mma_w(true, f_ok);
    if (abort) break;
    fresh = false;
    if (SV) aphase ^= 1u;  // every buffer of this tile was waited for
    // ---- hand dfeat (D_hi + 2^-11 D_lo, binary32) to the scatter warps through DF[b] ----
    const int b = jt & 1;
    int drained = 0;
    if (t == 0 && jt >= 2) drained = tc::mbar_wait_or_abort(empty + b, ((jt >> 1) - 1) & 1, abort_flag);
    if (t == 0 && drained == 2) atomicOr(&st_rw->status, kStatusTimeout);
    // the last layer's weight gradients: their operands (X0, the last delta) are rewritten by the
    // next tile
    bool okw = true;
    while (okw && w_waited != w_issued) okw = wait_w_next();
    tc::fence_after_sync();
    abort = tc::bar_or(kChainBar, TT, drained != 0 || !okw);
    if (abort) break;
    const int c0 = ch * 16;
    if (c0 < IN) {
      float df[16], dfl[16];
      tc::ld16(trow + c0, df);
      tc::ld16(trow + Y::C_DL + c0, dfl);
      tc::wait_ld();
      float *dst = dfbuf + (b * TM + r) * Y::DFS + c0;
#pragma unroll
      for (int i = 0; i < 16; i += 4)
        if (c0 + i < IN)
          *reinterpret_cast<float4 *>(dst + i) =
              make_float4(fmaf(dfl[i], kLoInv, df[i]), fmaf(dfl[i + 1], kLoInv, df[i + 1]),
                          fmaf(dfl[i + 2], kLoInv, df[i + 2]), fmaf(dfl[i + 3], kLoInv, df[i + 3]));
    }
    if (t == 0) {
      int64_t nv = (slot_end < r1 ? slot_end : r1) - ts;
      nv = nv < 0 ? 0 : (nv > TM ? TM : nv);
      info[b] = TileInfo{ts, slot, (int32_t)nv};
    }
    tc::mbar_arrive(full + b);
    ++jt;
    tc::fence_before_sync();
    tc::bar_sync(kChainBar, TT);
    tc::fence_after_sync();
  }

  if (abort) {
    if (t == 0) atomicOr(&st_rw->status, kStatusTimeout);
    *abort_flag = 1;             // releases scatter warps waiting for a tile
    tc::mbar_wait(mbar, phase);  // bounded: let any MMA still in flight finish before freeing TMEM
    // bounded: weight-gradient MMAs still in flight (one phase per commit, waited in order)
    while (BWD && w_waited != w_issued && wait_w_next()) {
    }
    // bounded: bulk copies still writing this CTA's shared memory land before it exits
    if (SV)
      for (int i = 0; i <= kGX0; ++i)
        if (a_pend & (1u << i)) tc::mbar_wait(abar + i, aphase);
  } else if (BWD && cur_slot >= 0) {
    flush(cur_slot);
  }
  }  // MMA / epilogue warps
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, Y::TCOLS);
}

// ---- forward with dedicated gather warps ---------------------------------------
// Four MMA / epilogue warps (one thread a tile row, both column halves) run one tile's MLP
// chain while eight gather warps (one thread a sample and level parity) interpolate the next
// tile's features into the other of two tensor-memory feature buffers (a gather warp writes the
// lanes of its 32 samples, as tcgen05.st requires): full[b] hands buffer b to the chain,
// and the commit of the layer-1 MMAs that read it (empty[b]) hands it back.  Two CTAs per SM
// keep two chains in flight.  Results are those of the forward above: the same per-level
// arithmetic, the same products (every layer reads A from tensor memory instead of shared memory).
constexpr int kWsMma = TM;                     // MMA / epilogue threads
constexpr int kWsGather = 2 * TM;              // gather threads
constexpr int kWsThreads = kWsMma + kWsGather;
constexpr uint32_t kGatherBar = 2;  // named barrier of the gather warps

template <int IN, bool VD>
struct LW {
  static constexpr int INP = L<IN, false, VD>::INP;
  static constexpr int CIN = L<IN, false, VD>::CIN;
  // every layer reads its input (high and low parts) from tensor memory: shared memory holds
  // only the weights (B operands), and no operand traffic competes with the table gathers
  // in the L1TEX data pipe
  static constexpr int W1 = 0;                  // weights, as in the layout above
  static constexpr int W2 = W1 + 64 * INP * 2;
  static constexpr int W3 = W2 + 64 * 64 * 2;
  static constexpr int V1 = W3 + 16 * 64 * 2;
  static constexpr int V2 = V1 + 64 * CIN * 2;
  static constexpr int V3 = V2 + 64 * 64 * 2;
  static constexpr int END = V3 + 16 * 64 * 2;
  // mbarriers (MMA commit, full[2], empty[2]), TMEM address, abort flag
  static constexpr int MISC = END;
  static constexpr int SMEM = MISC + 64;
  // tensor-memory columns: accumulator high parts 0..63, low parts C_DL..; a layer's output as the
  // next layer's A operand, high parts from A_HI, low parts from A_LO (32 columns: K <= 64); the
  // two feature buffers (layer 1's A operand) from F0, buffer b's high parts at F0 + 32 b, low
  // parts 16 columns further (K = INP <= 32); level l's two features are column l
  static constexpr uint32_t TCOLS = 256, C_DL = 64, A_HI = 128, A_LO = 160, F0 = 192;
  static_assert(INP <= 32, "feature buffers of 16 columns");
};

template <int IN, int G, bool COL, bool VD, int KL>
__global__ void __launch_bounds__(kWsThreads, 2) k_field_fws(const FieldArgs a) {
  constexpr int NM = kWsMma, NG = kWsGather;
  using Y = LW<IN, VD>;
  using A = L<IN, false, VD>;  // stored-activation offsets
  constexpr int INP = Y::INP;
  constexpr int CIN = Y::CIN;
  constexpr int ACT = A::act_bytes(COL);
  extern __shared__ __align__(1024) uint8_t sm[];
  uint64_t *mbar = reinterpret_cast<uint64_t *>(sm + Y::MISC);
  uint64_t *full = mbar + 1;   // [2] the gather warps filled feature buffer b
  uint64_t *empty = mbar + 3;  // [2] the layer-1 MMAs that read feature buffer b completed
  uint32_t *tslot = reinterpret_cast<uint32_t *>(sm + Y::MISC + 40);
  volatile int *abort_flag = reinterpret_cast<volatile int *>(sm + Y::MISC + 48);
  const int t = threadIdx.x, warp = t >> 5, lane = t & 31;
  const int r = 32 * (warp & 3) + lane;  // TMEM lane = tile row of an MMA / epilogue thread
  const snk_state *st = a.state;
  snk_state *st_rw = const_cast<snk_state *>(a.state);
  const ModelDev &m = a.m;
  const GridParams &gp = m.grid;
  const uint32_t s0 = tc::smem_u32(sm);

  if (t == 0) {
    tc::mbar_init(mbar, 1);
    for (int b = 0; b < 2; ++b) {
      tc::mbar_init(full + b, NG);
      tc::mbar_init(empty + b, 1);
    }
    *abort_flag = 0;
    tc::fence_mbar_init();
  }
  if (warp == 0) tc::tmem_alloc(tslot, Y::TCOLS);
  for (int i = t; i < Y::END / 16; i += blockDim.x) reinterpret_cast<uint4 *>(sm)[i] = make_uint4(0, 0, 0, 0);
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  const uint32_t tmem = *tslot;
  const uint32_t trow = tmem + ((uint32_t)(32 * (warp & 3)) << 16);

  int64_t r0 = 0, r1 = st->slot_base[kMaxSlots];
  if (a.slot_only >= 0) {
    r0 = st->slot_base[a.slot_only];
    r1 = r0 + st->slot_count[a.slot_only];
  }
  if (r1 > a.S) r1 = a.S;
  const int64_t n_tiles = r1 > r0 ? (r1 - r0 + TM - 1) / TM : 0;

  if (t >= NM) {
    // ---- gather warps: tile j's features into buffer j & 1 ----
    const int s = (t - NM) % TM, lq = (t - NM) / TM;  // sample of the tile, level parity
    constexpr int LS = NG / TM;                        // level groups (2)
    const uint64_t keep = l2_keep();                   // the tables stay in L2
    // this thread's lane of the feature buffers: the padding columns of layer 1's K (features
    // IN .. INP-1) are zero once and for all
    if (lq == 0 && IN < INP) {
      for (int b = 0; b < 2; ++b)
        for (int c = IN / 2; c < INP / 2; ++c) {
          tc::st1(trow + Y::F0 + 32 * b + c, 0u);
          tc::st1(trow + Y::F0 + 32 * b + 16 + c, 0u);
        }
    }
    int j = 0;
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      const int64_t ts = r0 + tile * TM;
      const int slot = slot_of(st, ts);
      if (slot < 0) continue;  // the MMA warps skip the same tiles
      const int b = j & 1;
      if (j >= 2) {
        // the layer-1 MMAs of tile j - 2 have read this buffer; every gather thread takes the
        // same branch (the named barrier below needs all of them)
        const int w = tc::mbar_wait_or_abort(empty + b, ((j >> 1) - 1) & 1, abort_flag);
        if (w == 2) {
          atomicOr(&st_rw->status, kStatusTimeout);
          *abort_flag = 1;
        }
        if (tc::bar_or(kGatherBar, NG, w != 0)) break;
        tc::fence_after_sync();  // the tensor-memory writes below follow the MMAs' reads
      }
      const uint32_t fh = trow + Y::F0 + 32 * b, fl = fh + 16;  // this warp's lanes of buffer b
      const int64_t slot_end = (int64_t)st->slot_base[slot] + st->slot_count[slot];
      const int64_t sidx = ts + s;
      const bool sval = sidx < slot_end && sidx < r1;
      float xyz[3] = {0.f, 0.f, 0.f};
      if (sval) {
#pragma unroll
        for (int q = 0; q < 3; ++q) xyz[q] = a.xyz[sidx * 3 + q];
      }
      const __half2 *tab0 = reinterpret_cast<const __half2 *>(a.params_lp + (int64_t)slot * m.tile_params);
      // KL levels per round: their corner loads are all issued before any is used
      for (int l0 = lq; l0 < gp.L; l0 += LS * KL) {
        __half2 hv[KL][8];
        float fr[KL][3];
#pragma unroll
        for (int k = 0; k < KL; ++k) {
          const int l = l0 + LS * k;
#pragma unroll
          for (int c = 0; c < 8; ++c) hv[k][c] = __float2half2_rn(0.f);
          fr[k][0] = fr[k][1] = fr[k][2] = 0.f;
          if (l < gp.L && sval) {
            if (a.cells_lp && gp.dense[l])  // one 32-byte load from the cell-major copy
              gather_cell(a.cells_lp + ((int64_t)slot * gp.n_cells + gp.cell_off[l]) * 16, xyz, gp.res[l], hv[k], fr[k], keep);
            else
              gather_corners(tab0 + gp.offset[l], xyz, gp.res[l], gp.dense[l] != 0, (uint32_t)gp.T - 1u, hv[k], fr[k],
                             keep);
          }
        }
#pragma unroll
        for (int k = 0; k < KL; ++k) {
          const int l = l0 + LS * k;
          if (l >= gp.L) break;
          const float2 f = interp_corners(hv[k], fr[k]);
          const float f0 = f.x, f1 = f.y;
          const uint32_t hp = pack_h2(f0, f1);
          const float2 hh = unpack_h2(hp);
          tc::st1(fh + l, hp);
          tc::st1(fl + l, pack_h2((f0 - hh.x) * kLoScale, (f1 - hh.y) * kLoScale));
        }
      }
      tc::wait_st();
      tc::fence_before_sync();
      tc::bar_sync(kGatherBar, NG);
      tc::fence_after_sync();
      // the tile's features, for the backward, in the shared-memory core layout the backward
      // copies them into: high parts (the level-parity-0 threads), and low parts (parity 1)
      // unless the activations are stored; each thread writes its sample's row
      if (lq == 0 || !a.acts) {
        uint16_t *ftile = a.feat_lp + (ts / TM) * (int64_t)(2 * TM * INP) + (lq ? TM * INP : 0);
        uint8_t *frow = reinterpret_cast<uint8_t *>(ftile);
#pragma unroll
        for (int c = 0; c < INP / 2; c += 8) {
          uint32_t v[8];
          tc::ld8((lq ? fl : fh) + c, v);
          tc::wait_ld();
          __stcs(reinterpret_cast<uint4 *>(frow + tc::core_off(s, 2 * c, TM)), make_uint4(v[0], v[1], v[2], v[3]));
          __stcs(reinterpret_cast<uint4 *>(frow + tc::core_off(s, 2 * c + 8, TM)), make_uint4(v[4], v[5], v[6], v[7]));
        }
      }
      tc::fence_before_sync();
      tc::mbar_arrive(full + b);
      ++j;
    }
  } else {
    // ---- MMA / epilogue warps ----
    uint32_t phase = 0;
    bool abort = false;
    int cur_slot = -1, j = 0;
    auto sync_mma = [&]() -> bool {
      const bool ok = tc::mbar_wait(mbar, phase);
      if (ok) phase ^= 1u;
      tc::fence_after_sync();
      return !tc::bar_or(kChainBar, NM, !ok);
    };
    // after an epilogue: its tensor-memory stores complete, shared-memory writes visible to the
    // tensor core, then the barrier
    auto handoff = [&]() {
      tc::wait_st();
      tc::fence_async_smem();
      tc::fence_before_sync();
      tc::bar_sync(kChainBar, NM);
      tc::fence_after_sync();
    };
    for (int64_t tile = blockIdx.x; tile < n_tiles; tile += gridDim.x) {
      const int64_t ts = r0 + tile * TM;
      const int slot = slot_of(st, ts);
      if (slot < 0) continue;
      if (slot != cur_slot) {
        tc::bar_sync(kChainBar, NM);
        const uint16_t *P = a.params_lp + (int64_t)slot * m.tile_params;
        const uint16_t *C = a.params_lp + m.colour_base + (m.shared_colour ? 0 : (int64_t)slot * m.colour_params);
        load_weights(sm + Y::W1, P + m.w1, 64, IN, 64, INP, NM);
        load_weights(sm + Y::W2, P + m.w2, 64, 64, 64, 64, NM);
        load_weights(sm + Y::W3, P + m.w3, G, 64, 16, 64, NM);
        if (COL) {
          load_weights(sm + Y::V1, C + m.v1, 64, VD ? CIN : G, 64, CIN, NM);
          load_weights(sm + Y::V2, C + m.v2, 64, 64, 64, 64, NM);
          load_weights(sm + Y::V3, C + m.v3, 3, 64, 16, 64, NM);
        }
        cur_slot = slot;
        handoff();
      }
      const int64_t slot_end = (int64_t)st->slot_base[slot] + st->slot_count[slot];
      const int64_t idx = ts + r;
      const bool valid = idx < slot_end && idx < r1;
      uint8_t *gact = a.acts ? reinterpret_cast<uint8_t *>(a.acts) + (ts / TM) * (int64_t)ACT : nullptr;
      const int b = j & 1;
      // the gather warps' features of this tile; the barrier also orders the last tile's
      // tensor-memory reads before this tile's MMAs
      {
        const int w = tc::mbar_wait_or_abort(full + b, (j >> 1) & 1, abort_flag);
        tc::fence_before_sync();
        abort = tc::bar_or(kChainBar, NM, w != 0);
        tc::fence_after_sync();
        if (abort) break;
      }
      const uint32_t fh = tmem + Y::F0 + 32 * b, fl = fh + 16;
      if (t == 0) {
        mma_fwd_ts<INP, 64>(tmem, fh, s0 + Y::W1);
        mma_fwd_ts<INP, 64>(tmem + Y::C_DL, fl, s0 + Y::W1);
        tc::commit(mbar);
        tc::commit(empty + b);
      }
      ++j;
      abort = !sync_mma();
      if (abort) break;
      for (int c = 0; c < 2; ++c)
        epi64_tm(trow, trow + Y::C_DL, trow + Y::A_HI, trow + Y::A_LO, r, c, gact ? gact + A::A1 : nullptr);
      handoff();
      if (t == 0) {
        mma_fwd_ts<64, 64>(tmem, tmem + Y::A_HI, s0 + Y::W2);
        mma_fwd_ts<64, 64>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::W2);
        tc::commit(mbar);
      }
      abort = !sync_mma();
      if (abort) break;
      for (int c = 0; c < 2; ++c)
        epi64_tm(trow, trow + Y::C_DL, trow + Y::A_HI, trow + Y::A_LO, r, c, gact ? gact + A::A2 : nullptr);
      handoff();
      if (t == 0) {
        mma_fwd_ts<64, 16>(tmem, tmem + Y::A_HI, s0 + Y::W3);
        mma_fwd_ts<64, 16>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::W3);
        tc::commit(mbar);
      }
      abort = !sync_mma();
      if (abort) break;
      float g[16];
      float rgb[3] = {0.f, 0.f, 0.f};
      ld16_pair(trow, trow + Y::C_DL, g);
      store16_tm(trow + Y::A_HI, trow + Y::A_LO, r, g, (COL && gact) ? gact + A::A3 : nullptr);
      if (!COL) {
#pragma unroll
        for (int k = 0; k < 3; ++k) rgb[k] = sigm(g[1 + k]);
      }
      if (VD) {
        // colour input columns 16..31: SH of the sample's ray direction
        float dir[3] = {0.f, 0.f, 1.f}, y[16];
        if (valid) {
          const uint32_t ray = a.smp_ray[idx];
#pragma unroll
          for (int q = 0; q < 3; ++q) dir[q] = a.ray_od[(int64_t)(3 + q) * a.n_rays + ray];
        }
        sh16(dir[0], dir[1], dir[2], y);
        store16_tm(trow + Y::A_HI + 8, trow + Y::A_LO + 8, r, y, gact ? gact + A::A3 + TM * 16 * 2 : nullptr);
      }
      handoff();
      if (COL) {
        if (t == 0) {
          mma_fwd_ts<CIN, 64>(tmem, tmem + Y::A_HI, s0 + Y::V1);
          mma_fwd_ts<CIN, 64>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::V1);
          tc::commit(mbar);
        }
        abort = !sync_mma();
        if (abort) break;
        for (int c = 0; c < 2; ++c)
        epi64_tm(trow, trow + Y::C_DL, trow + Y::A_HI, trow + Y::A_LO, r, c, gact ? gact + A::A4 : nullptr);
        handoff();
        if (t == 0) {
          mma_fwd_ts<64, 64>(tmem, tmem + Y::A_HI, s0 + Y::V2);
          mma_fwd_ts<64, 64>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::V2);
          tc::commit(mbar);
        }
        abort = !sync_mma();
        if (abort) break;
        for (int c = 0; c < 2; ++c)
        epi64_tm(trow, trow + Y::C_DL, trow + Y::A_HI, trow + Y::A_LO, r, c, gact ? gact + A::A5 : nullptr);
        handoff();
        if (t == 0) {
          mma_fwd_ts<64, 16>(tmem, tmem + Y::A_HI, s0 + Y::V3);
          mma_fwd_ts<64, 16>(tmem + Y::C_DL, tmem + Y::A_LO, s0 + Y::V3);
          tc::commit(mbar);
        }
        abort = !sync_mma();
        if (abort) break;
        float o[16];
        ld16_pair(trow, trow + Y::C_DL, o);
#pragma unroll
        for (int k = 0; k < 3; ++k) rgb[k] = sigm(o[k]);
      }
      if (valid)
        reinterpret_cast<float4 *>(a.sigma_rgb)[idx] = make_float4(__expf(g[0]), rgb[0], rgb[1], rgb[2]);
    }
    if (abort) {
      if (t == 0) atomicOr(&st_rw->status, kStatusTimeout);
      *abort_flag = 1;             // releases gather warps waiting for a buffer
      tc::mbar_wait(mbar, phase);  // bounded: let any MMA still in flight finish before freeing TMEM
    }
  }
  tc::fence_before_sync();
  __syncthreads();
  tc::fence_after_sync();
  if (warp == 0) tc::tmem_dealloc(tmem, Y::TCOLS);
}

template <int IN, int G, bool COL, bool VD, int KL>
cudaError_t launch_ws(const FieldArgs &a, int sm_count, cudaStream_t st) {
  using Y = LW<IN, VD>;
  static_assert(2 * (Y::SMEM + 1024) <= 233472, "two CTAs per SM: shared memory");
  static_assert(2 * Y::TCOLS <= 512, "two CTAs per SM: tensor memory");
  static_assert(Y::W1 % 16 == 0 && Y::MISC % 8 == 0, "alignment");
  auto k = k_field_fws<IN, G, COL, VD, KL>;
  static std::atomic<uint32_t> attr_done{0};  // per instantiation: devices whose limit is set
  if (cudaError_t e = set_smem_limit(k, Y::SMEM, attr_done); e != cudaSuccess) return e;
  const int64_t max_tiles = (a.S + TM - 1) / TM;
  int64_t grid = (int64_t)sm_count * 2;
  if (grid > max_tiles) grid = max_tiles;
  if (grid <= 0) return cudaSuccess;
  k<<<(unsigned)grid, kWsThreads, Y::SMEM, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <int IN, int G, bool COL, bool BWD, bool Q8, int KL, bool VD, int MINB, bool SV = false>
cudaError_t launch_t(const FieldArgs &a, int sm_count, cudaStream_t st, int fwd_ctas) {
  using Y = L<IN, BWD, VD>;
  static_assert(Y::SMEM <= 232448, "shared memory per CTA");
  static_assert(MINB * (Y::SMEM + 1024) <= 233472, "resident CTAs per SM: shared memory");
  static_assert(MINB * Y::TCOLS <= 512, "resident CTAs per SM: tensor memory");
  static_assert(Y::C_V1 + Y::CIN <= Y::C_DL || !BWD, "tensor-memory columns of dV1");
  static_assert(Y::MISC % 8 == 0 && 96 <= Y::SMEM - Y::MISC, "mbarriers and tile info in the MISC block");
  static_assert(Y::X0 % 16 == 0 && Y::X1 % 16 == 0 && Y::X3 % 16 == 0 && Y::X5 % 16 == 0, "bulk-copy targets");
  auto k = k_field_tc<IN, G, COL, BWD, Q8, KL, VD, MINB, SV>;
  static std::atomic<uint32_t> attr_done{0};  // per instantiation: devices whose limit is set
  if (cudaError_t e = set_smem_limit(k, Y::SMEM, attr_done); e != cudaSuccess) return e;
  const int64_t max_tiles = (a.S + TM - 1) / TM;
  const int per_sm = BWD ? 1 : fwd_ctas;
  int64_t grid = (int64_t)sm_count * per_sm;
  if (grid > max_tiles) grid = max_tiles;
  if (grid <= 0) return cudaSuccess;
  k<<<(unsigned)grid, BWD ? TT + scatter_threads(SV) : TT, Y::SMEM, st>>>(a);
  count_launches(1);
  return cudaGetLastError();
}

template <int IN, int G, bool COL, bool Q8, bool VD>
cudaError_t launch_mode(const FieldArgs &a, int sm_count, cudaStream_t st, const Tuning &tu) {
  if (a.mode == kBackward) {
    // stored activations (a training forward wrote them) or the forward recomputed
    if (a.acts) return launch_t<IN, G, COL, true, Q8, 1, VD, 1, true>(a, sm_count, st, 1);
    return launch_t<IN, G, COL, true, Q8, 1, VD, 1, false>(a, sm_count, st, 1);
  }
  // dedicated gather warps (the E4M3 forward reads its features: nothing to gather)
  if constexpr (!Q8) {
    if (tu.tc_fwd_split) {
      if (tu.tc_fwd_levels == 2) return launch_ws<IN, G, COL, VD, 2>(a, sm_count, st);
      return launch_ws<IN, G, COL, VD, 1>(a, sm_count, st);
    }
  }
  // three CTAs per SM: compiled for at most 85 registers a thread
  if (tu.tc_fwd_ctas == 3) {
    if (!Q8 && tu.tc_fwd_levels == 2) return launch_t<IN, G, COL, false, Q8, 2, VD, 3>(a, sm_count, st, 3);
    return launch_t<IN, G, COL, false, Q8, 1, VD, 3>(a, sm_count, st, 3);
  }
  // the E4M3 forward reads its features instead of gathering them: no gather shape to pick
  if (!Q8 && tu.tc_fwd_levels == 2)
    return launch_t<IN, G, COL, false, Q8, 2, VD, 2>(a, sm_count, st, tu.tc_fwd_ctas);
  return launch_t<IN, G, COL, false, Q8, 1, VD, 2>(a, sm_count, st, tu.tc_fwd_ctas);
}

template <int IN, int G, bool COL>
cudaError_t launch_q(const FieldArgs &a, int sm_count, cudaStream_t st, const Tuning &tu) {
  if constexpr (COL) {
    if (a.m.view_dirs) {
      if (a.m.e4m3 || a.smp_ray == nullptr || a.ray_od == nullptr || a.n_rays < 1) return cudaErrorInvalidValue;
      return launch_mode<IN, G, COL, false, true>(a, sm_count, st, tu);
    }
  }
  if (a.m.e4m3) return launch_mode<IN, G, COL, true, false>(a, sm_count, st, tu);
  return launch_mode<IN, G, COL, false, false>(a, sm_count, st, tu);
}

template <int IN>
cudaError_t launch_in(const FieldArgs &a, int sm_count, cudaStream_t st, const Tuning &tu) {
  if (a.m.colour) return launch_q<IN, 16, true>(a, sm_count, st, tu);
  return launch_q<IN, 4, false>(a, sm_count, st, tu);
}

}  // namespace

int64_t act_tile_bytes(bool colour, bool view_dirs) {
  return view_dirs ? L<32, true, true>::act_bytes(colour) : L<32, true, false>::act_bytes(colour);
}

cudaError_t launch_field_tc(const FieldArgs &a, int sm_count, cudaStream_t st, const Tuning &tu) {
  if (a.mode == kEncodeOnly || a.feat_lp == nullptr || a.params_lp == nullptr) return cudaErrorInvalidValue;
  if (a.m.e4m3 && (a.feat32 == nullptr || a.codes == nullptr || a.amax == nullptr)) return cudaErrorInvalidValue;
  switch (a.m.in_dim) {
    case 8: return launch_in<8>(a, sm_count, st, tu);
    case 16: return launch_in<16>(a, sm_count, st, tu);
    case 32: return launch_in<32>(a, sm_count, st, tu);
    default: return cudaErrorInvalidValue;
  }
}

}  // namespace snk
