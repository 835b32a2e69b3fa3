#pragma once
// Device code of the stabilizer-tensor-network simulation (sm_103a), shared by
// the translation units that instantiate it for complex64 (engine_f32.cu) and
// complex128 (engine_f64.cu), and by the allocation-free SVD
// (engine_noalloc.cu).
//
// One persistent CTA per shot slot walks the op list of a program segment
// (one syndrome round).  Clifford gates and Pauli noise update the inverse
// tableau held in shared memory (bit-exact integer row operations, Sec. IV A).
// A crosstalk rotation or a measurement pushes its Pauli through the tableau
// and acts on the shot's MPS as a bond-2 Pauli-string MPO; the touched span
// is then recompressed (Sec. IV B, Eq. 8) by a two-pass sweep:
//   left sweep   R_{k+1} = R factor of (R_k A'_k), R_a = identity since the
//                sites left of the span are left-canonical (Householder QR,
//                no Q formed); ||R_b A'_b||^2 is the squared norm of the new
//                state, which for a projector is the Born probability;
//   right sweep  C = R_k M_k = U Sigma V^dag (one-sided Jacobi); the kept
//                columns of V give the new right-canonical site and
//                M_{k-1} = A'_{k-1} (M_k V_keep) carries the rest to the left.
// Sigma holds the Schmidt values of the bond, so keeping the largest ones is
// the truncation of Eq. 8.  Small bonds are decomposed in shared memory (in
// double precision on the complex64 path where that fits); large bonds take
// the Householder R factor of C and run Jacobi on its conjugate transpose,
// which converges in a few sweeps.  Dense work runs in complex T (float or
// double); norms, Born probabilities and log-probabilities in double.
#include <cuda_runtime.h>
#include <math.h>

#include "../../include/stn.h"
#include "engine.h"

namespace stn {

// ---------------------------------------------------------------------------
// complex arithmetic
template <typename T>
struct cplx {
  T re, im;
};
template <typename T>
__device__ __forceinline__ cplx<T> cmake(T r, T i) {
  cplx<T> c;
  c.re = r;
  c.im = i;
  return c;
}
template <typename T>
__device__ __forceinline__ cplx<T> cadd(cplx<T> a, cplx<T> b) {
  return cmake<T>(a.re + b.re, a.im + b.im);
}
template <typename T>
__device__ __forceinline__ cplx<T> cmul(cplx<T> a, cplx<T> b) {
  return cmake<T>(a.re * b.re - a.im * b.im, a.re * b.im + a.im * b.re);
}
template <typename T>
__device__ __forceinline__ cplx<T> cconj(cplx<T> a) {
  return cmake<T>(a.re, -a.im);
}
template <typename T>
__device__ __forceinline__ cplx<T> cscale(cplx<T> a, T s) {
  return cmake<T>(a.re * s, a.im * s);
}
// acc += a * b
template <typename T>
__device__ __forceinline__ void cfma(cplx<T> &acc, cplx<T> a, cplx<T> b) {
  acc.re = fma(a.re, b.re, acc.re);
  acc.re = fma(-a.im, b.im, acc.re);
  acc.im = fma(a.re, b.im, acc.im);
  acc.im = fma(a.im, b.re, acc.im);
}
template <typename T>
__device__ __forceinline__ T cabs2(cplx<T> a) {
  return a.re * a.re + a.im * a.im;
}
// |a|^2 in double from double components: in single precision the square of
// a component below about 1e-19 is a denormal or zero, which would make the
// norm of a tiny vector (and a reflector built from it) inaccurate.
template <typename T>
__device__ __forceinline__ double cabs2d(cplx<T> a) {
  const double re = static_cast<double>(a.re), im = static_cast<double>(a.im);
  return re * re + im * im;
}
// i^m
template <typename T>
__device__ __forceinline__ cplx<T> ipow(int m) {
  m &= 3;
  return m == 0 ? cmake<T>(1, 0) : m == 1 ? cmake<T>(0, 1) : m == 2 ? cmake<T>(-1, 0) : cmake<T>(0, -1);
}

template <typename T>
struct Eps;
template <>
struct Eps<float> {
  static constexpr float v = 5.96e-8f;
};
template <>
struct Eps<double> {
  static constexpr double v = 1.11e-16;
};

// Complex elements of shared memory for the one-sided Jacobi SVD (the matrix
// and its right singular vectors); larger problems run on global scratch.
template <typename T>
struct SvdSmem;
template <>
struct SvdSmem<float> {
  static constexpr int elems = 22528;
};
template <>
struct SvdSmem<double> {
  static constexpr int elems = 8192;
};
constexpr int kMaxVec = 1024;  // longest Householder vector (4 * largest bond)

constexpr int kBM = 64, kBN = 64, kBK = 16, kPad = 4;

// ---------------------------------------------------------------------------
// Philox4x32-10 (Salmon, Moraes, Dror, Shaw, SC'11): two 32x32->64-bit
// multiplies per round, Weyl key schedule, ten rounds.
static __device__ __forceinline__ double philox_uniform(uint64_t seed, uint64_t shot, uint32_t ev) {
  uint32_t c0 = static_cast<uint32_t>(shot), c1 = static_cast<uint32_t>(shot >> 32);
  uint32_t c2 = ev, c3 = 0u;
  uint32_t k0 = static_cast<uint32_t>(seed), k1 = static_cast<uint32_t>(seed >> 32);
#pragma unroll
  for (int r = 0; r < 10; ++r) {
    uint32_t lo0 = 0xD2511F53u * c0, hi0 = __umulhi(0xD2511F53u, c0);
    uint32_t lo1 = 0xCD9E8D57u * c2, hi1 = __umulhi(0xCD9E8D57u, c2);
    uint32_t n0 = hi1 ^ c1 ^ k0, n2 = hi0 ^ c3 ^ k1;
    c0 = n0;
    c1 = lo1;
    c2 = n2;
    c3 = lo0;
    k0 += 0x9E3779B9u;
    k1 += 0xBB67AE85u;
  }
  uint64_t bits = (static_cast<uint64_t>(c0) << 21) ^ static_cast<uint64_t>(c1 >> 11);
  return static_cast<double>(bits) * 0x1.0p-53;
}


// ---------------------------------------------------------------------------
// CTA-wide helpers
static __device__ __forceinline__ int tid() { return threadIdx.x; }

// Sum of one double per thread over the CTA: a shuffle reduction per warp,
// then every thread adds the warps' partial sums (red: kThreads doubles of
// smem, of which the first kThreads / 32 are used).  Two barriers.
static __device__ double block_sum(double v, double *red) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = v;
  __syncthreads();
  double r = 0.0;
#pragma unroll
  for (int w = 0; w < kThreads / 32; ++w) r += red[w];
  __syncthreads();
  return r;
}

// ---------------------------------------------------------------------------
// Complex64 GEMM on the fifth-generation tensor cores (tcgen05).  The CTA's
// tensor-memory accumulator (128 lanes x 128 FP32 columns: the real part of
// a 128 x 64 output tile, then its imaginary part), the two mbarriers the
// MMAs complete on and the shared-memory staging area of the operand tiles
// live in g_tc; a kernel that allocates the accumulator sets enabled.
//
// Each product is FP32-accurate from TF32 operands by the 3-term split
// (Ootomo and Yokota, 2022): x = x_hi + x_lo with both parts TF32, and
// A B ~ A_hi B_hi + A_hi B_lo + A_lo B_hi.  The complex product takes four
// real ones, Re C = Re A Re B + Im A (-Im B) and Im C = Re A Im B + Im A Re B,
// so every k step of 8 issues 6 MMAs per part (M = 128, N = 64, K = 8,
// kind::tf32) accumulated in FP32; the negated imaginary part is staged on
// the smaller B tile.  The k range goes in chunks of 16: the 128 x 16 A tile
// (4 arrays: Re and Im, head and tail) and the 64 x 16 B tile (6 arrays:
// Re, Im and -Im, head and tail) of a chunk are written to one of two
// staging buffers in the no-swizzle K-major core-matrix layout (core
// matrices of 8 rows x 16 bytes, 128 bytes apart along k, 512 bytes apart
// between 8-row groups), each thread storing whole 16-byte core-matrix rows
// so that a quarter warp fills one core matrix without bank conflicts.  After
// a proxy fence one thread issues the chunk's 24 MMAs and commits them to the
// buffer's mbarrier, and the CTA stages the next chunk into the other buffer
// while they run; a buffer is refilled only after a bounded wait on its
// barrier (on time-out the CTA's status becomes STN_ETIMEOUT and the product
// is abandoned).
struct TcState {
  uint64_t bar[2];  // mbarriers of the two staging buffers
  uint32_t tmem;    // tensor-memory address of the accumulator
  uint32_t phase;   // bit b: parity of bar[b]'s next completion
  int enabled;      // the kernel allocated tensor memory and staging space
  int failed;       // a bounded wait ran out
  float *stage;     // two staging buffers of kTcBufFloats floats
};
static __shared__ __align__(8) TcState g_tc;

constexpr int kTcM = 128, kTcN = 64, kTcK = 16;
constexpr int kTcAFloats = kTcM * kTcK, kTcBFloats = kTcN * kTcK;
constexpr int kTcBufFloats = 4 * kTcAFloats + 6 * kTcBFloats;
constexpr int kTcStageFloats = 2 * kTcBufFloats;
constexpr uint32_t kTcCols = 2 * kTcN;
constexpr long long kTcWaitLimit = 1ll << 24;
// kind::tf32, FP32 accumulator, both operands K-major, N = 64, M = 128
constexpr uint32_t kTcIdesc = (1u << 4) | (2u << 7) | (2u << 10) | (static_cast<uint32_t>(kTcN >> 3) << 17) |
                              (static_cast<uint32_t>(kTcM >> 4) << 24);

__device__ __forceinline__ uint32_t smem_u32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// TF32 rounding (round to nearest, ties away) of an FP32 value, returned as
// the FP32 number it represents.
__device__ __forceinline__ float tf32_round(float x) {
  uint32_t r;
  asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(r) : "f"(x));
  return __uint_as_float(r);
}

// Float offset of the 16-byte core-matrix row (row, k = 4 kg .. 4 kg + 3)
// of a row x kTcK tile.
__device__ __forceinline__ int tc_row_offset(int row, int kg) {
  return (((row >> 3) * (kTcK / 4) + kg) * 128 + (row & 7) * 16) >> 2;
}

// Descriptor of the 8-wide k slice q of a staged tile (version 1, no
// swizzle): leading byte offset 128 (the next core matrix along k), stride
// byte offset kTcK / 4 x 128 (the next 8-row group).
__device__ __forceinline__ uint64_t tc_desc(const float *tile, int q) {
  const uint32_t a = smem_u32(tile) + static_cast<uint32_t>(q) * 256u;
  return static_cast<uint64_t>((a >> 4) & 0x3FFF) | (static_cast<uint64_t>(128 >> 4) << 16) |
         (static_cast<uint64_t>((kTcK / 4 * 128) >> 4) << 32) | (static_cast<uint64_t>(1) << 46);
}

__device__ __forceinline__ void tc_mma(uint32_t d, uint64_t a, uint64_t b, uint32_t acc) {
  asm volatile(
      "{\n\t.reg .pred p;\n\t"
      "setp.ne.b32 p, %4, 0;\n\t"
      "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n"
      :
      : "r"(d), "l"(a), "l"(b), "r"(kTcIdesc), "r"(acc));
}

__device__ __forceinline__ bool tc_wait(uint32_t bar, uint32_t phase) {
  for (long long it = 0; it < kTcWaitLimit; ++it) {
    uint32_t done;
    asm volatile(
        "{\n\t.reg .pred p;\n\t"
        "mbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(bar), "r"(phase)
        : "memory");
    if (done) return true;
  }
  return false;
}

// Tensor memory and barriers of a CTA that runs tensor-core GEMMs (CTA-wide;
// warp 0 allocates).  stage: kTcStageFloats floats of shared memory, 16-byte
// aligned, free whenever a GEMM runs.
static __device__ void tc_setup(float *stage) {
  if ((threadIdx.x >> 5) == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;\n" ::"r"(smem_u32(&g_tc.tmem)),
                 "r"(kTcCols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;\n");
  }
  if (threadIdx.x == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&g_tc.bar[0])));
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;\n" ::"r"(smem_u32(&g_tc.bar[1])));
    asm volatile("fence.mbarrier_init.release.cluster;\n" ::: "memory");
    g_tc.phase = 0;
    g_tc.failed = 0;
    g_tc.stage = stage;
    g_tc.enabled = 1;
  }
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
}

static __device__ void tc_teardown() {
  asm volatile("tcgen05.fence::before_thread_sync;\n");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;\n");
  if ((threadIdx.x >> 5) == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;\n" ::"r"(g_tc.tmem), "r"(kTcCols));
}

// Static shared memory starts with whatever the SM's previous kernel left
// there, so a kernel without tensor memory clears both flags.
static __device__ __forceinline__ void tc_disable() {
  if (threadIdx.x == 0) {
    g_tc.enabled = 0;
    g_tc.failed = 0;
  }
  __syncthreads();
}

static_assert(kThreads == 512, "the tensor-core staging and epilogue map 512 threads onto the tiles");

__device__ __forceinline__ void st_f4(float *p, float a, float b, float c, float d) {
  *reinterpret_cast<float4 *>(p) = make_float4(a, b, c, d);
}

// Stages the k chunk k0 .. k0 + kTcK - 1 of rows i0 .. i0 + 127 of op(A) and
// columns j0 .. j0 + 63 of op(B) into the staging buffer buf (zero outside
// the matrices).  Item f of a tile is the core-matrix row (row, kg) with
// row = (f & 7) + 8 (f >> 5) and kg = (f >> 3) & 3, so that the eight
// threads of a quarter warp write the eight rows of one core matrix.
template <int TA, int TB>
static __device__ __forceinline__ void tc_stage(float *buf, int M, int N, int K, const cplx<float> *A, int lda,
                                                const cplx<float> *B, int ldb, int i0, int j0, int k0) {
  for (int e = threadIdx.x; e < 4 * (kTcM + kTcN); e += kThreads) {
    const bool isA = e < 4 * kTcM;  // warp-uniform: 4 kTcM is a multiple of kThreads
    const int f = isA ? e : e - 4 * kTcM;
    const int row = (f & 7) | ((f >> 5) << 3), kg = (f >> 3) & 3;
    float rh[4], rl[4], ih[4], il[4];
#pragma unroll
    for (int u = 0; u < 4; ++u) {
      const int gk = k0 + 4 * kg + u;
      cplx<float> v = cmake<float>(0.f, 0.f);
      if (isA) {
        const int gi = i0 + row;
        if (gi < M && gk < K)
          v = TA == 0 ? A[static_cast<int64_t>(gi) * lda + gk] : cconj(A[static_cast<int64_t>(gk) * lda + gi]);
      } else {
        const int gj = j0 + row;
        if (gj < N && gk < K)
          v = TB == 0 ? B[static_cast<int64_t>(gk) * ldb + gj] : cconj(B[static_cast<int64_t>(gj) * ldb + gk]);
      }
      rh[u] = tf32_round(v.re);
      rl[u] = tf32_round(v.re - rh[u]);
      ih[u] = tf32_round(v.im);
      il[u] = tf32_round(v.im - ih[u]);
    }
    const int o = tc_row_offset(row, kg);
    float *dst = isA ? buf + o : buf + 4 * kTcAFloats + o;
    const int s = isA ? kTcAFloats : kTcBFloats;
    st_f4(dst, rh[0], rh[1], rh[2], rh[3]);
    st_f4(dst + s, rl[0], rl[1], rl[2], rl[3]);
    st_f4(dst + 2 * s, ih[0], ih[1], ih[2], ih[3]);
    st_f4(dst + 3 * s, il[0], il[1], il[2], il[3]);
    if (!isA) {
      st_f4(dst + 4 * s, -ih[0], -ih[1], -ih[2], -ih[3]);
      st_f4(dst + 5 * s, -il[0], -il[1], -il[2], -il[3]);
    }
  }
}

// The 24 MMAs of one staged chunk (two k slices of 8) into the real and
// imaginary accumulators; the first slice of a tile overwrites them.
static __device__ __forceinline__ void tc_issue_chunk(const float *buf, uint32_t tm_re, uint32_t tm_im, bool first) {
  const float *Ab = buf, *Bb = buf + 4 * kTcAFloats;
#pragma unroll
  for (int q = 0; q < kTcK / 8; ++q) {
    const uint32_t acc = (!first || q > 0) ? 1u : 0u;
    const uint64_t a_rh = tc_desc(Ab, q), a_rl = tc_desc(Ab + kTcAFloats, q), a_ih = tc_desc(Ab + 2 * kTcAFloats, q),
                   a_il = tc_desc(Ab + 3 * kTcAFloats, q);
    const uint64_t b_rh = tc_desc(Bb, q), b_rl = tc_desc(Bb + kTcBFloats, q), b_ih = tc_desc(Bb + 2 * kTcBFloats, q),
                   b_il = tc_desc(Bb + 3 * kTcBFloats, q), b_nh = tc_desc(Bb + 4 * kTcBFloats, q),
                   b_nl = tc_desc(Bb + 5 * kTcBFloats, q);
    tc_mma(tm_re, a_rh, b_rh, acc);  // Re A Re B
    tc_mma(tm_re, a_rh, b_rl, 1u);
    tc_mma(tm_re, a_rl, b_rh, 1u);
    tc_mma(tm_re, a_ih, b_nh, 1u);   // Im A (-Im B)
    tc_mma(tm_re, a_ih, b_nl, 1u);
    tc_mma(tm_re, a_il, b_nh, 1u);
    tc_mma(tm_im, a_rh, b_ih, acc);  // Re A Im B
    tc_mma(tm_im, a_rh, b_il, 1u);
    tc_mma(tm_im, a_rl, b_ih, 1u);
    tc_mma(tm_im, a_ih, b_rh, 1u);   // Im A Re B
    tc_mma(tm_im, a_ih, b_rl, 1u);
    tc_mma(tm_im, a_il, b_rh, 1u);
  }
}

// Kept out of line so that its registers do not weigh on the callers'.
template <int TA, int TB>
static __device__ __noinline__ void cgemm_tc(int M, int N, int K, cplx<float> alpha, const cplx<float> *A, int lda,
                                             const cplx<float> *B, int ldb, cplx<float> beta, cplx<float> *C,
                                             int ldc) {
  float *st = g_tc.stage;
  const uint32_t tm_re = g_tc.tmem, tm_im = g_tc.tmem + kTcN;
  const uint32_t bar0 = smem_u32(&g_tc.bar[0]), bar1 = smem_u32(&g_tc.bar[1]);
  uint32_t phase = g_tc.phase;
  const int warp = threadIdx.x >> 5, lane = threadIdx.x & 31;
  const bool beta0 = beta.re == 0.f && beta.im == 0.f;
  const int nk = (K + kTcK - 1) / kTcK;
  bool ok = true;
  uint32_t pending = 0;  // bit b: buffer b holds committed MMAs not yet waited on
  for (int i0 = 0; i0 < M && ok; i0 += kTcM) {
    for (int j0 = 0; j0 < N && ok; j0 += kTcN) {
      for (int kc = 0; kc < nk; ++kc) {
        const int b = kc & 1;
        bool waited = true;
        if (pending & (1u << b)) {  // the MMAs of chunk kc - 2 still read this buffer
          waited = tc_wait(b ? bar1 : bar0, (phase >> b) & 1u);
          phase ^= 1u << b;
          pending &= ~(1u << b);
        }
        float *buf = st + b * kTcBufFloats;
        if (waited) tc_stage<TA, TB>(buf, M, N, K, A, lda, B, ldb, i0, j0, kc * kTcK);
        asm volatile("fence.proxy.async.shared::cta;\n" ::: "memory");
        asm volatile("tcgen05.fence::before_thread_sync;\n");
        const int failed = __syncthreads_or(waited ? 0 : 1);
        asm volatile("tcgen05.fence::after_thread_sync;\n");
        if (failed) {
          ok = false;
          break;
        }
        if (threadIdx.x == 0) {
          tc_issue_chunk(buf, tm_re, tm_im, kc == 0);
          asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];\n" ::"r"(
                           b ? bar1 : bar0)
                       : "memory");
        }
        pending |= 1u << b;
      }
      if (!ok) break;
      // the tile's last MMAs (and the older chunk in the other buffer)
      bool waited = true;
#pragma unroll
      for (int b = 0; b < 2; ++b)
        if (pending & (1u << b)) {
          waited = tc_wait(b ? bar1 : bar0, (phase >> b) & 1u) && waited;
          phase ^= 1u << b;
        }
      pending = 0;
      asm volatile("tcgen05.fence::after_thread_sync;\n");
      if (__syncthreads_or(waited ? 0 : 1)) {
        ok = false;
        break;
      }
      // epilogue: warp w reads lanes 32 (w % 4) .. + 31, columns 16 (w / 4) .. + 15,
      // eight at a time
      const int quarter = warp & 3;
      const uint32_t lane_off = static_cast<uint32_t>(32 * quarter) << 16;
      const int row = i0 + 32 * quarter + lane;
#pragma unroll
      for (int half = 0; half < 2; ++half) {
        const int cb = 16 * (warp >> 2) + 8 * half;
        uint32_t vr[8], vi[8];
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                     : "=r"(vr[0]), "=r"(vr[1]), "=r"(vr[2]), "=r"(vr[3]), "=r"(vr[4]), "=r"(vr[5]), "=r"(vr[6]),
                       "=r"(vr[7])
                     : "r"(tm_re + lane_off + cb));
        asm volatile("tcgen05.ld.sync.aligned.32x32b.x8.b32 {%0,%1,%2,%3,%4,%5,%6,%7}, [%8];\n"
                     : "=r"(vi[0]), "=r"(vi[1]), "=r"(vi[2]), "=r"(vi[3]), "=r"(vi[4]), "=r"(vi[5]), "=r"(vi[6]),
                       "=r"(vi[7])
                     : "r"(tm_im + lane_off + cb));
        asm volatile("tcgen05.wait::ld.sync.aligned;\n" ::: "memory");
        if (row < M) {
#pragma unroll
          for (int c = 0; c < 8; ++c) {
            const int col = j0 + cb + c;
            if (col >= N) continue;
            cplx<float> v = cmul(alpha, cmake<float>(__uint_as_float(vr[c]), __uint_as_float(vi[c])));
            cplx<float> *dst = &C[static_cast<int64_t>(row) * ldc + col];
            if (!beta0) v = cadd(v, cmul(beta, *dst));
            *dst = v;
          }
        }
      }
      asm volatile("tcgen05.fence::before_thread_sync;\n");
      __syncthreads();
      asm volatile("tcgen05.fence::after_thread_sync;\n");
    }
  }
  if (!ok) {  // give the MMAs in flight a last bounded chance to land, then report
#pragma unroll
    for (int b = 0; b < 2; ++b)
      if (pending & (1u << b)) {
        tc_wait(b ? bar1 : bar0, (phase >> b) & 1u);
        phase ^= 1u << b;
      }
    if (threadIdx.x == 0) g_tc.failed = 1;
  }
  if (threadIdx.x == 0) g_tc.phase = phase;
  __syncthreads();
}

// C = alpha * op(A) op(B) + beta * C, all row-major, op = identity (0) or
// conjugate transpose (1).  op(A) is M x K, op(B) is K x N.  Complex64
// products large enough to fill the tensor-core tiles run cgemm_tc when the
// kernel enabled it; the rest (and complex128) run on the CUDA cores below.
template <typename T, int TA, int TB>
static __device__ void cgemm(int M, int N, int K, cplx<T> alpha, const cplx<T> *A, int lda,
                      const cplx<T> *B, int ldb, cplx<T> beta, cplx<T> *C, int ldc,
                      cplx<T> *tile) {
  if constexpr (sizeof(T) == 4) {
    if (g_tc.enabled && M >= 64 && N >= 32 && K >= kTcK) {
      cgemm_tc<TA, TB>(M, N, K, alpha, A, lda, B, ldb, beta, C, ldc);
      return;
    }
  }
  // thread (ty, tx) of a kTY x 16 grid owns rows ty + kTY a (a < kMR) and
  // columns tx + 16 b (b < 4) of the 64 x 64 output tile
  constexpr int kTY = kThreads / 16, kMR = kBM / kTY;
  static_assert(kMR * kTY == kBM && (kBM * kBK) % kThreads == 0, "tile shape");
  cplx<T> *As = tile;                    // [kBK][kBM + kPad]
  cplx<T> *Bs = tile + kBK * (kBM + kPad);  // [kBK][kBN + kPad]
  const int ty = tid() / 16, tx = tid() % 16;
  const int tilesM = (M + kBM - 1) / kBM, tilesN = (N + kBN - 1) / kBN;
  for (int t = 0; t < tilesM * tilesN; ++t) {
    const int i0 = (t / tilesN) * kBM, j0 = (t % tilesN) * kBN;
    cplx<T> acc[kMR][4];
#pragma unroll
    for (int a = 0; a < kMR; ++a)
#pragma unroll
      for (int b = 0; b < 4; ++b) acc[a][b] = cmake<T>(0, 0);
    for (int k0 = 0; k0 < K; k0 += kBK) {
      // A tile: element (i, k) of op(A)
#pragma unroll
      for (int r = 0; r < (kBM * kBK) / kThreads; ++r) {
        int e = tid() + r * kThreads;
        int i, k;
        if (TA == 0) { k = e % kBK; i = e / kBK; } else { i = e % kBM; k = e / kBM; }
        int gi = i0 + i, gk = k0 + k;
        cplx<T> v = cmake<T>(0, 0);
        if (gi < M && gk < K) v = TA == 0 ? A[static_cast<int64_t>(gi) * lda + gk]
                                          : cconj(A[static_cast<int64_t>(gk) * lda + gi]);
        As[k * (kBM + kPad) + i] = v;
      }
#pragma unroll
      for (int r = 0; r < (kBN * kBK) / kThreads; ++r) {
        int e = tid() + r * kThreads;
        int j, k;
        if (TB == 0) { j = e % kBN; k = e / kBN; } else { k = e % kBK; j = e / kBK; }
        int gj = j0 + j, gk = k0 + k;
        cplx<T> v = cmake<T>(0, 0);
        if (gj < N && gk < K) v = TB == 0 ? B[static_cast<int64_t>(gk) * ldb + gj]
                                          : cconj(B[static_cast<int64_t>(gj) * ldb + gk]);
        Bs[k * (kBN + kPad) + j] = v;
      }
      __syncthreads();
#pragma unroll
      for (int k = 0; k < kBK; ++k) {
        cplx<T> av[kMR], bv[4];
#pragma unroll
        for (int a = 0; a < kMR; ++a) av[a] = As[k * (kBM + kPad) + ty + kTY * a];
#pragma unroll
        for (int b = 0; b < 4; ++b) bv[b] = Bs[k * (kBN + kPad) + tx + 16 * b];
#pragma unroll
        for (int a = 0; a < kMR; ++a)
#pragma unroll
          for (int b = 0; b < 4; ++b) cfma(acc[a][b], av[a], bv[b]);
      }
      __syncthreads();
    }
#pragma unroll
    for (int a = 0; a < kMR; ++a) {
      int gi = i0 + ty + kTY * a;
      if (gi >= M) continue;
#pragma unroll
      for (int b = 0; b < 4; ++b) {
        int gj = j0 + tx + 16 * b;
        if (gj >= N) continue;
        cplx<T> *c = &C[static_cast<int64_t>(gi) * ldc + gj];
        cplx<T> v = cmul(alpha, acc[a][b]);
        if (beta.re != T(0) || beta.im != T(0)) v = cadd(v, cmul(beta, *c));
        *c = v;
      }
    }
  }
  __syncthreads();
}

static __device__ __forceinline__ int warp_id() { return threadIdx.x >> 5; }
static __device__ __forceinline__ int lane_id() { return threadIdx.x & 31; }
constexpr int kWarps = kThreads / 32;

template <typename T>
__device__ __forceinline__ T warp_sum(T v) {
#pragma unroll
  for (int o = 16; o > 0; o >>= 1) v += __shfl_xor_sync(0xffffffffu, v, o);
  return v;
}

// Householder QR of B (m x n, row-major, leading dimension ld), in place: on
// return rows 0..min(m,n)-1 hold R (upper trapezoidal) and the rest is zero.
// Each step uses the Hermitian reflector P = I - 2 u u^dag with
// P x = gamma e_1, gamma = -(x_0/|x_0|) ||x||.  Blocked by panels of nb
// columns: a panel is copied to shared memory (pbuf) and factored there,
// its reflectors u_1..u_nb are kept as the columns of V, and the product
// P_nb ... P_1 = I - V T^dag V^dag (compact WY form, T upper triangular with
// T_kk = 2, T[0:k, k] = -2 T[0:k, 0:k] V[:, 0:k]^dag u_k) is applied to the
// trailing columns at once, one thread per column, so the trailing matrix is
// read and written twice per panel rather than per column.  pbuf needs
// m (nb + 1) + 2 nb^2 complex elements (nb is reduced to fit).  CTA-wide.
constexpr int kQrPanel = 16;

static __device__ __forceinline__ int qr_panel_width(int m, int pbuf_elems) {
  int nb = kQrPanel;
  while (nb > 1 && static_cast<int64_t>(m) * (nb + 1) + 2 * nb * nb > pbuf_elems) --nb;
  return nb;
}

// T of the compact WY form of a panel's reflectors (columns of Vp, row-major
// [mr][ldv], u_b zero above row b): T upper triangular, T_kk = 2,
// T[0:k, k] = -2 T[0:k, 0:k] (V[:, 0:k]^dag u_k).  G is scratch.  CTA-wide.
template <typename T>
static __device__ void wy_t_factor(int mr, int jb, int nb, int ldv, const cplx<T> *Vp, cplx<T> *Tm, cplx<T> *G) {
  for (int pr = warp_id(); pr < jb * jb; pr += kWarps) {
    const int a = pr / jb, b = pr % jb;
    if (a >= b) continue;
    T gr = 0, gi = 0;
    for (int i = b + lane_id(); i < mr; i += 32) {  // u_b vanishes above row b
      const cplx<T> x = Vp[i * ldv + a], y = Vp[i * ldv + b];
      gr += x.re * y.re + x.im * y.im;
      gi += x.re * y.im - x.im * y.re;
    }
    gr = warp_sum(gr);
    gi = warp_sum(gi);
    if (lane_id() == 0) G[a * nb + b] = cmake<T>(gr, gi);
  }
  __syncthreads();
  if (tid() == 0) {
    for (int k = 0; k < jb; ++k) {
      Tm[k * nb + k] = cmake<T>(2, 0);
      for (int a = 0; a < k; ++a) {
        cplx<T> acc = cmake<T>(0, 0);
        for (int b = a; b < k; ++b) cfma(acc, Tm[a * nb + b], G[b * nb + k]);
        Tm[a * nb + k] = cscale(acc, T(-2));
      }
    }
  }
  __syncthreads();
}

// With vstore (row-major m x min(m,n)), the reflectors are also kept there
// (column j holds u_j in rows j..m-1; rows above are not written) so that
// form_q can build Q explicitly.
template <typename T>
static __device__ void qr_r_inplace(int m, int n, cplx<T> *B, int ld, cplx<T> *pbuf, int pbuf_elems, double *red,
                             double *dm, cplx<T> *vstore = nullptr) {
  const int steps = min(m, n);
  const int nb = qr_panel_width(m, pbuf_elems);
  // rows of the panel padded to an odd number of elements, so that a column
  // walked by consecutive threads spreads over the shared-memory banks
  const int ldv = nb + 1;
  cplx<T> *Vp = pbuf;                                    // [(m - j0)][ldv], row-major
  cplx<T> *Tm = pbuf + static_cast<int64_t>(m) * ldv;  // [nb][nb]
  cplx<T> *G = Tm + nb * nb;                            // [nb][nb], G[a][b] = u_a^dag u_b
  for (int j0 = 0; j0 < steps; j0 += nb) {
    const int jb = min(nb, steps - j0);
    const int mr = m - j0;
    for (int e = tid(); e < mr * jb; e += kThreads) {
      const int i = e / jb, c = e % jb;
      Vp[i * ldv + c] = B[static_cast<int64_t>(j0 + i) * ld + j0 + c];
    }
    __syncthreads();
    for (int jj = 0; jj < jb; ++jj) {
      double nx2 = 0;
      for (int i = jj + tid(); i < mr; i += kThreads) nx2 += cabs2d(Vp[i * ldv + jj]);
      nx2 = block_sum(nx2, red);
      // rows above the diagonal of this column are final R entries
      for (int i = tid(); i < jj; i += kThreads) B[static_cast<int64_t>(j0 + i) * ld + j0 + jj] = Vp[i * ldv + jj];
      if (!(nx2 > 1e-60)) {  // (numerically) zero column: no reflector, R row jj is final
        for (int i = tid(); i < mr; i += kThreads) {
          if (i >= jj) B[static_cast<int64_t>(j0 + i) * ld + j0 + jj] = cmake<T>(0, 0);
          Vp[i * ldv + jj] = cmake<T>(0, 0);
        }
        __syncthreads();
        continue;
      }
      if (tid() == 0) {
        cplx<T> al = Vp[jj * ldv + jj];
        double aa = sqrt(cabs2d(al));
        double nx = sqrt(nx2);
        double pr = aa > 0 ? al.re / aa : 1.0, pi = aa > 0 ? al.im / aa : 0.0;
        dm[0] = -pr * nx;  // gamma
        dm[1] = -pi * nx;
        dm[2] = 1.0 / sqrt(2.0 * nx * (nx + aa));  // 1 / ||x - gamma e_1||
      }
      __syncthreads();
      const cplx<T> gam = cmake<T>(static_cast<T>(dm[0]), static_cast<T>(dm[1]));
      const T sc = static_cast<T>(dm[2]);
      for (int i = tid(); i < mr; i += kThreads) {
        cplx<T> u = cmake<T>(0, 0);
        if (i >= jj) {
          cplx<T> x = Vp[i * ldv + jj];
          if (i == jj) x = cmake<T>(x.re - gam.re, x.im - gam.im);
          u = cscale(x, sc);
          B[static_cast<int64_t>(j0 + i) * ld + j0 + jj] = i == jj ? gam : cmake<T>(0, 0);
        }
        Vp[i * ldv + jj] = u;
      }
      __syncthreads();
      // the rest of the panel: b <- b - 2 u (u^dag b), one warp per column
      for (int c = jj + 1 + warp_id(); c < jb; c += kWarps) {
        T sr = 0, si = 0;
        for (int i = jj + lane_id(); i < mr; i += 32) {
          const cplx<T> u = Vp[i * ldv + jj], b = Vp[i * ldv + c];
          sr += u.re * b.re + u.im * b.im;
          si += u.re * b.im - u.im * b.re;
        }
        sr = __shfl_sync(0xffffffffu, warp_sum(sr), 0);
        si = __shfl_sync(0xffffffffu, warp_sum(si), 0);
        const cplx<T> s2 = cmake<T>(T(2) * sr, T(2) * si);
        for (int i = jj + lane_id(); i < mr; i += 32) {
          const cplx<T> t = cmul(Vp[i * ldv + jj], s2);
          cplx<T> &b = Vp[i * ldv + c];
          b = cmake<T>(b.re - t.re, b.im - t.im);
        }
      }
      __syncthreads();
    }
    if (vstore != nullptr)
      for (int e = tid(); e < mr * jb; e += kThreads) {
        const int i = e / jb, c = e % jb;
        vstore[static_cast<int64_t>(j0 + i) * steps + j0 + c] = Vp[i * ldv + c];
      }
    if (j0 + jb >= n) {  // no trailing columns
      __syncthreads();
      continue;
    }
    wy_t_factor<T>(mr, jb, nb, ldv, Vp, Tm, G);
    // trailing columns: b <- b - V (T^dag (V^dag b)).  The nt trailing
    // columns go to the warps in groups of cpw = 32 / ns consecutive columns
    // (coalesced row reads), and the ns lanes that share a column split its
    // rows (rows s, s + ns, s + 2 ns, ... for slice s); their partials of
    // w = V^dag b are summed by shuffles, so that a trailing matrix of a few
    // hundred columns still occupies the whole CTA.  Rows go four at a time
    // so that four loads per thread are in flight.
    {
      const int nt = n - j0 - jb;
      int ns = 1;
      while (ns < 8 && nt * 2 * ns <= kThreads) ns *= 2;
      const int cpw = 32 / ns, s = lane_id() / cpw;
      for (int cb = j0 + jb + warp_id() * cpw; cb < n; cb += kWarps * cpw) {  // warp-uniform trip count
        const int c = cb + lane_id() % cpw;
        const bool valid = c < n;
        cplx<T> w[kQrPanel];
#pragma unroll
        for (int k = 0; k < kQrPanel; ++k) w[k] = cmake<T>(0, 0);
        if (valid) {
          int i = s;
          for (; i + 3 * ns < mr; i += 4 * ns) {
            cplx<T> b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = B[static_cast<int64_t>(j0 + i + u * ns) * ld + c];
#pragma unroll
            for (int u = 0; u < 4; ++u)
#pragma unroll
              for (int k = 0; k < kQrPanel; ++k)
                if (k < jb) cfma(w[k], cconj(Vp[(i + u * ns) * ldv + k]), b[u]);
          }
          for (; i < mr; i += ns) {
            const cplx<T> b = B[static_cast<int64_t>(j0 + i) * ld + c];
#pragma unroll
            for (int k = 0; k < kQrPanel; ++k)
              if (k < jb) cfma(w[k], cconj(Vp[i * ldv + k]), b);
          }
        }
        for (int off = cpw; off < 32; off *= 2)
#pragma unroll
          for (int k = 0; k < kQrPanel; ++k)
            if (k < jb) {
              w[k].re += __shfl_xor_sync(0xffffffffu, w[k].re, off);
              w[k].im += __shfl_xor_sync(0xffffffffu, w[k].im, off);
            }
        // w <- T^dag w in place, highest index first: w'[a] = sum_{b<=a} conj(T[b][a]) w[b]
#pragma unroll
        for (int a = kQrPanel - 1; a >= 0; --a) {
          if (a >= jb) continue;
          cplx<T> acc = cmake<T>(0, 0);
#pragma unroll
          for (int b = 0; b <= a; ++b) cfma(acc, cconj(Tm[b * nb + a]), w[b]);
          w[a] = acc;
        }
        if (valid) {
          int i = s;
          for (; i + 3 * ns < mr; i += 4 * ns) {
            cplx<T> b[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) b[u] = B[static_cast<int64_t>(j0 + i + u * ns) * ld + c];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
#pragma unroll
              for (int k = 0; k < kQrPanel; ++k)
                if (k < jb) {
                  const cplx<T> t = cmul(Vp[(i + u * ns) * ldv + k], w[k]);
                  b[u] = cmake<T>(b[u].re - t.re, b[u].im - t.im);
                }
              B[static_cast<int64_t>(j0 + i + u * ns) * ld + c] = b[u];
            }
          }
          for (; i < mr; i += ns) {
            cplx<T> &bref = B[static_cast<int64_t>(j0 + i) * ld + c];
            cplx<T> acc = bref;
#pragma unroll
            for (int k = 0; k < kQrPanel; ++k)
              if (k < jb) {
                const cplx<T> t = cmul(Vp[i * ldv + k], w[k]);
                acc = cmake<T>(acc.re - t.re, acc.im - t.im);
              }
            bref = acc;
          }
        }
      }
    }
    __syncthreads();
  }
}

// Explicit Q (m x steps, row-major) of a Householder QR whose reflectors
// qr_r_inplace kept in vstore: Q = P_1 ... P_steps [I; 0], built panel by
// panel from the last, each panel applied as I - V T V^dag to the columns at
// or right of it (the columns left of panel p are unit vectors its
// reflectors do not touch).  Same shared-memory needs as qr_r_inplace.
template <typename T>
static __device__ void form_q(int m, int steps, const cplx<T> *vstore, cplx<T> *Q, cplx<T> *pbuf, int pbuf_elems) {
  const int nb = qr_panel_width(m, pbuf_elems);
  const int ldv = nb + 1;
  cplx<T> *Vp = pbuf;
  cplx<T> *Tm = pbuf + static_cast<int64_t>(m) * ldv;
  cplx<T> *G = Tm + nb * nb;
  for (int64_t e = tid(); e < static_cast<int64_t>(m) * steps; e += kThreads) {
    const int i = static_cast<int>(e / steps), c = static_cast<int>(e % steps);
    Q[e] = cmake<T>(i == c ? T(1) : T(0), 0);
  }
  const int npan = (steps + nb - 1) / nb;
  for (int p = npan - 1; p >= 0; --p) {
    const int j0 = p * nb, jb = min(nb, steps - j0), mr = m - j0;
    for (int e = tid(); e < mr * nb; e += kThreads) {
      const int i = e / nb, c = e % nb;
      // u_c is zero above its own row; rows above were never written
      Vp[i * ldv + c] = (c < jb && i >= c) ? vstore[static_cast<int64_t>(j0 + i) * steps + j0 + c] : cmake<T>(0, 0);
    }
    __syncthreads();
    wy_t_factor<T>(mr, jb, nb, ldv, Vp, Tm, G);
    for (int c = j0 + tid(); c < steps; c += kThreads) {
      cplx<T> w[kQrPanel];
#pragma unroll
      for (int k = 0; k < kQrPanel; ++k) w[k] = cmake<T>(0, 0);
      int i = 0;
      for (; i + 4 <= mr; i += 4) {
        cplx<T> q[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) q[u] = Q[static_cast<int64_t>(j0 + i + u) * steps + c];
#pragma unroll
        for (int u = 0; u < 4; ++u)
#pragma unroll
          for (int k = 0; k < kQrPanel; ++k)
            if (k < jb) cfma(w[k], cconj(Vp[(i + u) * ldv + k]), q[u]);
      }
      for (; i < mr; ++i) {
        const cplx<T> q = Q[static_cast<int64_t>(j0 + i) * steps + c];
#pragma unroll
        for (int k = 0; k < kQrPanel; ++k)
          if (k < jb) cfma(w[k], cconj(Vp[i * ldv + k]), q);
      }
      // w <- T w in place, lowest index first: w'[a] = sum_{b>=a} T[a][b] w[b]
#pragma unroll
      for (int a = 0; a < kQrPanel; ++a) {
        if (a >= jb) continue;
        cplx<T> acc = cmake<T>(0, 0);
#pragma unroll
        for (int b = a; b < kQrPanel; ++b)
          if (b < jb) cfma(acc, Tm[a * nb + b], w[b]);
        w[a] = acc;
      }
      for (int i = 0; i < mr; ++i) {
        cplx<T> &qref = Q[static_cast<int64_t>(j0 + i) * steps + c];
        cplx<T> acc = qref;
#pragma unroll
        for (int k = 0; k < kQrPanel; ++k)
          if (k < jb) {
            const cplx<T> t = cmul(Vp[i * ldv + k], w[k]);
            acc = cmake<T>(acc.re - t.re, acc.im - t.im);
          }
        qref = acc;
      }
    }
    __syncthreads();
  }
}

// One-sided (Hestenes) Jacobi SVD.  Columns of C (m x n, column-major,
// leading dimension m) are rotated pairwise until mutually orthogonal, so
// that C V = U diag(sigma); V (column-major) accumulates the rotations unless
// it is null (then only the rotated columns, U diag(sigma), are wanted).
// Round-robin ordering, one warp per column pair, the pairs of a round are
// disjoint.  A pair is left alone when its columns are orthogonal to the
// rounding level of their dot products, or when one column is negligible
// (norm at the rounding level of ||C||: no information, and its dot products
// would underflow).

// One sweep over all column pairs of C (ldc = m) with V (n x n, ld = ldv).
// Sets *flag when a rotation happened.  CTA-wide.
template <typename T>
static __device__ void onesided_sweep(int m, int n, cplx<T> *C, cplx<T> *V, int ldv, T tol, T negligible,
                               int *flag) {
  const int mm = n + (n & 1);
  const int half = mm / 2;
  for (int round = 0; round < mm - 1; ++round) {
    for (int pi = warp_id(); pi < half; pi += kWarps) {
      int p, q;
      if (pi == 0) { p = mm - 1; q = round; }
      else { p = (round + pi) % (mm - 1); q = (round - pi + (mm - 1)) % (mm - 1); }
      if (p > q) { int t = p; p = q; q = t; }
      if (q >= n) continue;
      cplx<T> *cp = C + static_cast<int64_t>(p) * m, *cq = C + static_cast<int64_t>(q) * m;
      T al = 0, be = 0, gr = 0, gi = 0;
      for (int i = lane_id(); i < m; i += 32) {
        cplx<T> x = cp[i], y = cq[i];
        al += cabs2(x);
        be += cabs2(y);
        gr += x.re * y.re + x.im * y.im;  // conj(x) y
        gi += x.re * y.im - x.im * y.re;
      }
      al = __shfl_sync(0xffffffffu, warp_sum(al), 0);
      be = __shfl_sync(0xffffffffu, warp_sum(be), 0);
      gr = __shfl_sync(0xffffffffu, warp_sum(gr), 0);
      gi = __shfl_sync(0xffffffffu, warp_sum(gi), 0);
      if (!(al > negligible) || !(be > negligible)) continue;
      T absg = sqrt(gr * gr + gi * gi);
      if (!(absg > tol * sqrt(al) * sqrt(be))) continue;
      T zeta = (be - al) / (T(2) * absg);
      T az = fabs(zeta);
      T t = az > T(1e10) ? T(0.5) / az : T(1) / (az + sqrt(T(1) + zeta * zeta));
      if (zeta < 0) t = -t;
      T cs = T(1) / sqrt(T(1) + t * t), sn = t * cs;
      cplx<T> uc = cmake<T>(gr / absg, -gi / absg);  // conj(gamma / |gamma|)
      for (int i = lane_id(); i < m; i += 32) {
        cplx<T> x = cp[i], y = cmul(uc, cq[i]);
        cp[i] = cmake<T>(cs * x.re - sn * y.re, cs * x.im - sn * y.im);
        cq[i] = cmake<T>(sn * x.re + cs * y.re, sn * x.im + cs * y.im);
      }
      if (V == nullptr) {
        if (lane_id() == 0) *flag = 1;
        continue;
      }
      cplx<T> *vp = V + static_cast<int64_t>(p) * ldv, *vq = V + static_cast<int64_t>(q) * ldv;
      for (int i = lane_id(); i < n; i += 32) {
        cplx<T> x = vp[i], y = cmul(uc, vq[i]);
        vp[i] = cmake<T>(cs * x.re - sn * y.re, cs * x.im - sn * y.im);
        vq[i] = cmake<T>(sn * x.re + cs * y.re, sn * x.im + cs * y.im);
      }
      if (lane_id() == 0) *flag = 1;
    }
    __syncthreads();
  }
}

template <typename T>
__device__ __forceinline__ T onesided_tol(int m) {
  return Eps<T>::v * T(4) * sqrt(static_cast<T>(m > 1 ? m : 1));
}

template <typename T>
static __device__ T onesided_prologue(int m, int n, const cplx<T> *C, cplx<T> *V, double *red) {
  for (int e = tid(); V != nullptr && e < n * n; e += kThreads) {
    int j = e / n, i = e % n;
    V[e] = cmake<T>(i == j ? T(1) : T(0), 0);
  }
  double fro2 = 0;
  for (int64_t e = tid(); e < static_cast<int64_t>(m) * n; e += kThreads) fro2 += cabs2d(C[e]);
  fro2 = block_sum(fro2, red);
  return static_cast<T>(static_cast<double>(Eps<T>::v) * static_cast<double>(Eps<T>::v) * fro2);
}

template <typename T>
static __device__ void onesided_epilogue(int m, int n, const cplx<T> *C, T *sig2) {
  for (int j = warp_id(); j < n; j += kWarps) {
    double a = 0;
    for (int i = lane_id(); i < m; i += 32) a += cabs2d(C[static_cast<int64_t>(j) * m + i]);
    a = warp_sum(a);
    if (lane_id() == 0) sig2[j] = static_cast<T>(a);
  }
  __syncthreads();
}

constexpr int kMaxSweepsF = 15, kMaxSweepsD = 20;
constexpr int kMaxBlockedSweepsF = 30, kMaxBlockedSweepsD = 40;

// Unblocked: C and V wherever they are (shared memory for small problems).
template <typename T>
static __device__ int svd_onesided(int m, int n, cplx<T> *C, cplx<T> *V, T *sig2, int *flag, double *red) {
  const T negligible = onesided_prologue<T>(m, n, C, V, red);
  const T tol = onesided_tol<T>(m);
  const int max_sweeps = sizeof(T) == 4 ? kMaxSweepsF : kMaxSweepsD;
  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps && n > 1; ++sweep) {
    ++sweeps;
    if (tid() == 0) *flag = 0;
    __syncthreads();
    onesided_sweep<T>(m, n, C, V, n, tol, negligible, flag);
    int f = *flag;
    __syncthreads();
    if (!f) break;
  }
  onesided_epilogue<T>(m, n, C, sig2);
  return sweeps;
}

// Blocked, for problems larger than shared memory: C (m x n, column-major)
// and V (n x n, or null) stay in global memory and the columns are split into
// blocks of bw.  One outer sweep first orthogonalises the columns inside every
// block, then lets every pair of blocks exchange its cross pairs: the block
// pairs of a tournament round are disjoint, and inside a block pair (I, J)
// step t rotates the disjoint column pairs (b, (b + t) mod w_a) over the
// smaller block's columns b and the larger block's columns, so each cross
// pair is visited once per sweep.  A visited block (or block pair) is staged
// in shared memory with its squared column norms, which the warp that rotates
// a pair recomputes from the rotated columns, so testing a pair costs one dot
// product.  With V, a w x w unitary Q accumulates the rotations of the visit
// and is applied to V's matching columns afterwards, a chunk of V's rows at a
// time through shared memory.  Outer sweeps repeat until one rotates nothing.
// Sum over the 16 lanes of a half warp (mask: those lanes), the same value
// broadcast to all of them.
template <typename T>
__device__ __forceinline__ T half_sum(T v, unsigned mask) {
#pragma unroll
  for (int o = 8; o > 0; o >>= 1) v += __shfl_xor_sync(mask, v, o, 16);
  return __shfl_sync(mask, v, 0, 16);
}

// One column pair (p, q) of a staged block, rotated by half a warp (the two
// halves of a warp work on two disjoint pairs).
template <typename T>
static __device__ void jacobi_rotate_staged(int m, int w, cplx<T> *Cb, cplx<T> *Q, T *nr, int p, int q, T tol,
                                     T negligible, int *flag) {
  const T al = nr[p], be = nr[q];
  if (!(al > negligible) || !(be > negligible)) return;
  const int hl = lane_id() & 15;
  const unsigned mask = 0xFFFFu << (lane_id() & 16);
  cplx<T> *cp = Cb + static_cast<int64_t>(p) * m, *cq = Cb + static_cast<int64_t>(q) * m;
  T gr = 0, gi = 0;
  for (int i = hl; i < m; i += 16) {
    cplx<T> x = cp[i], y = cq[i];
    gr += x.re * y.re + x.im * y.im;  // conj(x) y
    gi += x.re * y.im - x.im * y.re;
  }
  gr = half_sum(gr, mask);
  gi = half_sum(gi, mask);
  const T absg = sqrt(gr * gr + gi * gi);
  if (!(absg > tol * sqrt(al) * sqrt(be))) return;
  const T zeta = (be - al) / (T(2) * absg);
  const T az = fabs(zeta);
  T t = az > T(1e10) ? T(0.5) / az : T(1) / (az + sqrt(T(1) + zeta * zeta));
  if (zeta < 0) t = -t;
  const T cs = T(1) / sqrt(T(1) + t * t), sn = t * cs;
  const cplx<T> uc = cmake<T>(gr / absg, -gi / absg);  // conj(gamma / |gamma|)
  T np = 0, nq = 0;
  for (int i = hl; i < m; i += 16) {
    cplx<T> x = cp[i], y = cmul(uc, cq[i]);
    cplx<T> xn = cmake<T>(cs * x.re - sn * y.re, cs * x.im - sn * y.im);
    cplx<T> yn = cmake<T>(sn * x.re + cs * y.re, sn * x.im + cs * y.im);
    cp[i] = xn;
    cq[i] = yn;
    np += cabs2(xn);
    nq += cabs2(yn);
  }
  np = half_sum(np, mask);
  nq = half_sum(nq, mask);
  if (Q != nullptr) {
    cplx<T> *qp = Q + static_cast<int64_t>(p) * w, *qq = Q + static_cast<int64_t>(q) * w;
    for (int i = hl; i < w; i += 16) {
      cplx<T> x = qp[i], y = cmul(uc, qq[i]);
      qp[i] = cmake<T>(cs * x.re - sn * y.re, cs * x.im - sn * y.im);
      qq[i] = cmake<T>(sn * x.re + cs * y.re, sn * x.im + cs * y.im);
    }
  }
  __syncwarp(mask);
  if (hl == 0) {
    nr[p] = np;
    nr[q] = nq;
    *flag = 1;
  }
}

// ---------------------------------------------------------------------------
// Register-resident cross visit of the blocked Jacobi SVD (complex64, no V).
// The two column blocks I and J (16 columns each, the last one possibly
// shorter and zero-padded) of C (m x n, column-major, m <= 256 R) are held in
// registers, thread t owning rows t, t + 256, ... of all 32 columns.  Step s
// (s = 0..15) rotates the 16 disjoint cross pairs (I_b, J_{(b+s) mod 16}):
// every thread forms its rows' contributions to the 16 complex dot products,
// one CTA-wide reduction sums them, 16 threads turn them into rotations
// (the same Hestenes rotation as onesided_sweep), and every thread applies
// them to its rows.  The J registers are then shifted by one slot, so the
// pairing stays slot b with slot b and all register indices are static.
// Column norms are reduced once per visit and then updated with the exact
// one-sided Jacobi identities |x'|^2 = |x|^2 - t|g|, |y'|^2 = |y|^2 + t|g|.
// Each column is read and written once per visit, instead of twice per pair.
// wrk: 8 * 32 + 64 + 32 floats of shared memory.  Returns whether any pair
// rotated (the columns are written back only then).

// Reduce-scatter of 32 values over a warp: lane l returns the warp sum of v[l].
__device__ __forceinline__ float warp_reduce_scatter32(float (&v)[32]) {
  const int lane = lane_id();
#pragma unroll
  for (int h = 16; h >= 1; h >>= 1) {
    const bool upper = (lane & h) != 0;
#pragma unroll
    for (int i = 0; i < h; ++i) {
      const float a = v[i], b = v[i + h];
      const float send = upper ? a : b;
      const float keep = upper ? b : a;
      v[i] = keep + __shfl_xor_sync(0xffffffffu, send, h);
    }
  }
  return v[0];
}

// CTA sum of 32 values per thread: thread i < 32 returns the sum of value i.
// Contains one barrier; red holds kWarps * 32 floats.
__device__ __forceinline__ float cta_reduce32(float (&v)[32], float *red) {
  const float s = warp_reduce_scatter32(v);
  red[warp_id() * 32 + lane_id()] = s;
  __syncthreads();
  float tot = 0.f;
  if (tid() < 32) {
#pragma unroll
    for (int w = 0; w < kWarps; ++w) tot += red[w * 32 + tid()];
  }
  return tot;
}

constexpr int kRvWrkFloats = kWarps * 32 + 64 + 32 + 4;
// sorted eigenvalues of a bond (at most 512) and, during an SVD, the
// register-visit reductions
constexpr int kLamElems = kRvWrkFloats > 512 ? kRvWrkFloats : 512;

template <int R>
static __device__ bool cross_visit_regs(int m, cplx<float> *C, int c0, int wI, int c1, int wJ, float tol,
                                        float negligible, float *wrk) {
  float *red = wrk;                   // kWarps * 32
  float4 *prm = reinterpret_cast<float4 *>(wrk + kWarps * 32);  // 16 rotations
  float *nrm = wrk + kWarps * 32 + 64;  // 32 column norms: I then J (in J's column order)
  int *rot = reinterpret_cast<int *>(nrm + 32);
  cplx<float> xi[R][16], xj[R][16];
  const int t = tid();
#pragma unroll
  for (int r = 0; r < R; ++r) {
    const int row = t + r * kThreads;
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      xi[r][b] = (row < m && b < wI) ? C[static_cast<int64_t>(c0 + b) * m + row] : cmake<float>(0.f, 0.f);
      xj[r][b] = (row < m && b < wJ) ? C[static_cast<int64_t>(c1 + b) * m + row] : cmake<float>(0.f, 0.f);
    }
  }
  {
    float v[32];
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      float a = 0.f, c = 0.f;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        a += cabs2(xi[r][b]);
        c += cabs2(xj[r][b]);
      }
      v[b] = a;
      v[16 + b] = c;
    }
    const float s = cta_reduce32(v, red);
    if (t < 32) nrm[t] = s;
    if (t == 0) *rot = 0;
  }
  __syncthreads();
  for (int step = 0; step < 16; ++step) {
    float v[32];
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      float gr = 0.f, gi = 0.f;
#pragma unroll
      for (int r = 0; r < R; ++r) {
        const cplx<float> x = xi[r][b], y = xj[r][b];
        gr += x.re * y.re + x.im * y.im;  // conj(x) y
        gi += x.re * y.im - x.im * y.re;
      }
      v[2 * b] = gr;
      v[2 * b + 1] = gi;
    }
    const float s = cta_reduce32(v, red);
    if (t < 32) {
      const float gi = __shfl_down_sync(0xffffffffu, s, 1);
      if ((t & 1) == 0) {
        const int b = t >> 1, jb = (b + step) & 15;
        const float gr = s, al = nrm[b], be = nrm[16 + jb];
        float4 p = make_float4(1.f, 0.f, 1.f, 0.f);  // identity: skipped
        if (al > negligible && be > negligible) {
          const float absg = sqrtf(gr * gr + gi * gi);
          if (absg > tol * sqrtf(al) * sqrtf(be)) {
            const float zeta = (be - al) / (2.f * absg);
            const float az = fabsf(zeta);
            float tt = az > 1e10f ? 0.5f / az : 1.f / (az + sqrtf(1.f + zeta * zeta));
            if (zeta < 0.f) tt = -tt;
            const float cs = 1.f / sqrtf(1.f + tt * tt), sn = tt * cs;
            p = make_float4(cs, sn, gr / absg, -gi / absg);  // conj(g / |g|)
            nrm[b] = fmaxf(al - tt * absg, 0.f);
            nrm[16 + jb] = fmaxf(be + tt * absg, 0.f);
            *rot = 1;
          }
        }
        prm[b] = p;
      }
    }
    __syncthreads();
#pragma unroll
    for (int b = 0; b < 16; ++b) {
      const float4 p = prm[b];
      if (p.x != 1.f || p.y != 0.f || p.z != 1.f || p.w != 0.f) {  // uniform over the CTA
        const cplx<float> uc = cmake<float>(p.z, p.w);
#pragma unroll
        for (int r = 0; r < R; ++r) {
          const cplx<float> x = xi[r][b], y = cmul(uc, xj[r][b]);
          xi[r][b] = cmake<float>(p.x * x.re - p.y * y.re, p.x * x.im - p.y * y.im);
          xj[r][b] = cmake<float>(p.y * x.re + p.x * y.re, p.y * x.im + p.x * y.im);
        }
      }
    }
    // slot b of J now pairs with I_b at the next step: shift J by one slot
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const cplx<float> first = xj[r][0];
#pragma unroll
      for (int b = 0; b < 15; ++b) xj[r][b] = xj[r][b + 1];
      xj[r][15] = first;
    }
  }
  __syncthreads();
  const bool rotated = *rot != 0;
  if (rotated) {
#pragma unroll
    for (int r = 0; r < R; ++r) {
      const int row = t + r * kThreads;
      if (row >= m) continue;
#pragma unroll
      for (int b = 0; b < 16; ++b) {
        if (b < wI) C[static_cast<int64_t>(c0 + b) * m + row] = xi[r][b];
        if (b < wJ) C[static_cast<int64_t>(c1 + b) * m + row] = xj[r][b];
      }
    }
  }
  __syncthreads();
  return rotated;
}

template <typename T>
static __device__ bool cross_visit_dispatch(int m, cplx<T> *C, int c0, int wI, int c1, int wJ, T tol, T negligible,
                                            float *wrk) {
  if constexpr (sizeof(T) == 4) {
    return cross_visit_regs<1>(m, C, c0, wI, c1, wJ, tol, negligible, wrk);  // m <= kThreads
  } else {
    return false;
  }
}

// rv_wrk (kRvWrkFloats floats of shared memory, or null): with it, a
// complex64 problem without V and with m <= kThreads visits block pairs
// with cross_visit_regs (blocks of 16 columns); the blocks alone are still
// staged in shared memory.
template <typename T>
static __device__ int svd_onesided_blocked(int m, int n, cplx<T> *C, cplx<T> *V, T *sig2, int *flag,
                                     double *red, cplx<T> *sbuf, int sbuf_elems, float *rv_wrk = nullptr) {
  const T negligible = onesided_prologue<T>(m, n, C, V, red);
  const T tol = onesided_tol<T>(m);
  // staged block pair: Q (w x w, only with V), norms (w complex slots),
  // columns (m x w)
  const bool withV = V != nullptr;
  const bool regs = sizeof(T) == 4 && !withV && rv_wrk != nullptr && m <= kThreads &&
                    static_cast<int64_t>(m) * 16 + 32 <= sbuf_elems;
  int bw = 32;
  while (bw > 1 && static_cast<int64_t>(m) * 2 * bw + (withV ? 4 * bw * bw : 0) + 2 * bw > sbuf_elems) --bw;
  if (bw > 2 * kWarps) bw -= bw % (2 * kWarps);  // whole waves of half warps per step
  if (regs) bw = 16;
  const int nb = (n + bw - 1) / bw, nbe = nb + (nb & 1);
  const int max_sweeps = sizeof(T) == 4 ? kMaxBlockedSweepsF : kMaxBlockedSweepsD;
  int *any = flag + 1;
  // Visits follow a fixed order (each block alone, then the tournament), so
  // visit v of sweep s has the stamp s * per_sweep + v.  last_mod[I] is the
  // stamp of the last visit that rotated columns of block I.  A visit whose
  // previous occurrence (one sweep earlier) rotated nothing, with neither
  // block changed since, would see the same columns and rotate nothing again:
  // it is skipped, which changes no result.  The stamps live in `red`, free
  // between the prologue and the epilogue.
  const int per_sweep = nb + (nbe - 1) * (nbe / 2);
  int *last_mod = reinterpret_cast<int *>(red);
  const bool skipping = nb <= static_cast<int>(kThreads * sizeof(double) / sizeof(int));
  if (skipping) {
    for (int i = tid(); i < nb; i += kThreads) last_mod[i] = -1;
    __syncthreads();
  }

  auto visit = [&](int I, int J, int stamp) {
    if (skipping && stamp >= per_sweep && last_mod[I] < stamp - per_sweep && last_mod[J] < stamp - per_sweep)
      return;
    const bool self = I == J;
    const int c0 = I * bw, wI = min(bw, n - c0);
    const int c1 = J * bw, wJ = self ? 0 : min(bw, n - c1);
    const int w = wI + wJ;
    if (regs && !self) {
      if (cross_visit_dispatch<T>(m, C, c0, wI, c1, wJ, tol, negligible, rv_wrk)) {
        if (skipping && tid() == 0) last_mod[I] = last_mod[J] = stamp;
        if (tid() == 0) *any = 1;
      }
      __syncthreads();
      return;
    }
    auto gcol = [&](int c) { return c < wI ? c0 + c : c1 + (c - wI); };
    const int qe = withV ? w * w : 0;
    cplx<T> *Q = withV ? sbuf : nullptr;
    T *nr = reinterpret_cast<T *>(sbuf + qe);
    cplx<T> *Cb = sbuf + qe + w;
    for (int e = tid(); e < m * w; e += kThreads) {
      const int c = e / m, i = e % m;
      Cb[e] = C[static_cast<int64_t>(gcol(c)) * m + i];
    }
    for (int e = tid(); e < qe; e += kThreads) Q[e] = cmake<T>((e / w) == (e % w) ? T(1) : T(0), 0);
    __syncthreads();
    for (int c = warp_id(); c < w; c += kWarps) {
      T a = 0;
      for (int i = lane_id(); i < m; i += 32) a += cabs2(Cb[static_cast<int64_t>(c) * m + i]);
      a = __shfl_sync(0xffffffffu, warp_sum(a), 0);
      if (lane_id() == 0) nr[c] = a;
    }
    if (tid() == 0) *flag = 0;
    __syncthreads();
    if (self) {
      const int mm = w + (w & 1), half = mm / 2;
      const int hw = 2 * warp_id() + (lane_id() >> 4);  // half-warp index
      for (int round = 0; round < mm - 1; ++round) {
        for (int pi = hw; pi < half; pi += 2 * kWarps) {
          int p, q;
          if (pi == 0) { p = mm - 1; q = round; }
          else { p = (round + pi) % (mm - 1); q = (round - pi + (mm - 1)) % (mm - 1); }
          if (p > q) { int tt = p; p = q; q = tt; }
          if (q >= w) continue;
          jacobi_rotate_staged<T>(m, w, Cb, Q, nr, p, q, tol, negligible, flag);
        }
        __syncthreads();
      }
    } else {
      const bool i_larger = wI >= wJ;
      const int wa = i_larger ? wI : wJ, wb = i_larger ? wJ : wI;
      const int hw = 2 * warp_id() + (lane_id() >> 4);  // half-warp index
      for (int t = 0; t < wa; ++t) {
        for (int b = hw; b < wb; b += 2 * kWarps) {
          const int a = (b + t) % wa;
          const int p = i_larger ? a : b, q = wI + (i_larger ? b : a);
          jacobi_rotate_staged<T>(m, w, Cb, Q, nr, p, q, tol, negligible, flag);
        }
        __syncthreads();
      }
    }
    const int rotated = *flag;
    __syncthreads();
    if (!rotated) return;
    if (skipping && tid() == 0) last_mod[I] = last_mod[J] = stamp;
    for (int e = tid(); e < m * w; e += kThreads) {
      const int c = e / m, i = e % m;
      C[static_cast<int64_t>(gcol(c)) * m + i] = Cb[e];
    }
    __syncthreads();
    // V[:, cols] <- V[:, cols] Q, rows staged in the column buffer
    const int rows_cap = (sbuf_elems - qe - w) / w;
    for (int i0 = 0; withV && i0 < n; i0 += rows_cap) {
      const int rows = min(rows_cap, n - i0);
      for (int e = tid(); e < rows * w; e += kThreads) {
        const int c = e / rows, i = e % rows;
        Cb[e] = V[static_cast<int64_t>(gcol(c)) * n + i0 + i];
      }
      __syncthreads();
      // four output columns per thread: one staged element feeds four FMAs
      const int groups = (w + 3) / 4;
      for (int e = tid(); e < rows * groups; e += kThreads) {
        const int g = e / rows, i = e % rows, cb = 4 * g;
        cplx<T> acc[4];
#pragma unroll
        for (int u = 0; u < 4; ++u) acc[u] = cmake<T>(0, 0);
        for (int j = 0; j < w; ++j) {
          const cplx<T> v = Cb[j * rows + i];
#pragma unroll
          for (int u = 0; u < 4; ++u)
            if (cb + u < w) cfma(acc[u], v, Q[(cb + u) * w + j]);
        }
#pragma unroll
        for (int u = 0; u < 4; ++u)
          if (cb + u < w) V[static_cast<int64_t>(gcol(cb + u)) * n + i0 + i] = acc[u];
      }
      __syncthreads();
    }
    if (tid() == 0) *any = 1;
  };

  int sweeps = 0;
  for (int sweep = 0; sweep < max_sweeps && n > 1; ++sweep) {
    ++sweeps;
    if (tid() == 0) *any = 0;
    __syncthreads();
    const int base = sweep * per_sweep;
    for (int I = 0; I < nb; ++I) visit(I, I, base + I);
    for (int round = 0; round < nbe - 1; ++round) {
      for (int bp = 0; bp < nbe / 2; ++bp) {
        int I, J;
        if (bp == 0) { I = nbe - 1; J = round; }
        else { I = (round + bp) % (nbe - 1); J = (round - bp + (nbe - 1)) % (nbe - 1); }
        if (I > J) { int tt = I; I = J; J = tt; }
        if (J >= nb) continue;
        visit(I, J, base + nb + round * (nbe / 2) + bp);
      }
    }
    __syncthreads();
    const int f = *any;
    __syncthreads();
    if (!f) break;
  }
  onesided_epilogue<T>(m, n, C, sig2);
  return sweeps;
}

// One Newton-Schulz step X <- X (3 I - X^dag X) / 2 on the k orthonormal-to-
// rounding columns of X (n x k, row-major, ld k): the accumulated rotations
// leave X orthonormal only to about sqrt(#rotations) eps; this brings it back
// to the rounding level of one product.  G and Y are k x k and n x k scratch.
template <typename T>
static __device__ void reorthonormalize(int n, int k, cplx<T> *X, cplx<T> *G, cplx<T> *Y, cplx<T> *tile) {
  const cplx<T> one = cmake<T>(1, 0), zero = cmake<T>(0, 0);
  cgemm<T, 1, 0>(k, k, n, one, X, k, X, k, zero, G, k, tile);
  for (int e = tid(); e < k * k; e += kThreads) {
    int i = e / k, j = e % k;
    cplx<T> g = G[e];
    G[e] = cmake<T>((i == j ? T(1.5) : T(0)) - T(0.5) * g.re, -T(0.5) * g.im);
  }
  __syncthreads();
  cgemm<T, 0, 0>(n, k, k, one, X, k, G, k, zero, Y, k, tile);
  for (int e = tid(); e < n * k; e += kThreads) X[e] = Y[e];
  __syncthreads();
}

// Descending order of lambda (ties by index): perm[rank] = index.
template <typename T>
static __device__ void sort_desc(int n, const T *lam, int *perm) {
  for (int i = tid(); i < n; i += kThreads) perm[i] = i;
  __syncthreads();
  for (int i = tid(); i < n; i += kThreads) {
    T li = lam[i];
    int rank = 0;
    for (int j = 0; j < n; ++j) {
      T lj = lam[j];
      rank += (lj > li) || (lj == li && j < i);
    }
    if (li == li && rank < n) perm[rank] = i;  // a NaN keeps the identity slot
  }
  __syncthreads();
}

// ---------------------------------------------------------------------------
// The MPO of one rotation or measurement.
// MPO_ADJ_B: the adjoint of a case-B measurement, U |v><0|_j (U the
// controlled-Pauli product of the measurement, |v> its site-j eigenvector).
enum MpoKind { MPO_ROT = 0, MPO_PROJ_Z = 1, MPO_PROJ_B = 2, MPO_ADJ_B = 3 };

template <typename T>
struct MpoSpec {
  int kind, lo, hi, j;
  int par;         // case A: parity of the Z support that the projector keeps
  cplx<T> w0, w1;  // branch weights (folded into site lo)
  cplx<T> v0, v1;  // measurement eigenvector at site j (case B)
};

// 2x2 operator (row-major op[s*2 + t]) of branch `br` at site k of the span.
template <typename T>
static __device__ void site_op(const MpoSpec<T> &sp, const uint64_t *ppx, const uint64_t *ppz, int k,
                        int br, cplx<T> op[4]) {
  const bool x = (ppx[k >> 6] >> (k & 63)) & 1, z = (ppz[k >> 6] >> (k & 63)) & 1;
  const cplx<T> zero = cmake<T>(0, 0), one = cmake<T>(1, 0);
  op[0] = one; op[1] = zero; op[2] = zero; op[3] = one;
  if (br == 1) {
    if (sp.kind == MPO_PROJ_B && k == sp.j) {
      op[0] = zero; op[1] = cconj(sp.v1); op[2] = zero; op[3] = zero;
    } else if (sp.kind == MPO_ADJ_B && k == sp.j) {  // v1 |1><0|
      op[0] = zero; op[1] = zero; op[2] = sp.v1; op[3] = zero;
    } else if (sp.kind == MPO_PROJ_B || sp.kind == MPO_ADJ_B) {
      // Hermitian letter of P' at k (controlled-Pauli target)
      if (x && !z) { op[0] = zero; op[1] = one; op[2] = one; op[3] = zero; }
      else if (x && z) { op[0] = zero; op[1] = cmake<T>(0, -1); op[2] = cmake<T>(0, 1); op[3] = zero; }
      else if (z) { op[3] = cmake<T>(-1, 0); }
    } else {
      // X^x Z^z (MPO_PROJ_Z has x = 0 on every site)
      if (x && !z) { op[0] = zero; op[1] = one; op[2] = one; op[3] = zero; }
      else if (x && z) { op[0] = zero; op[1] = cmake<T>(-1, 0); op[2] = one; op[3] = zero; }
      else if (z) { op[3] = cmake<T>(-1, 0); }
    }
  } else if (sp.kind == MPO_PROJ_B && k == sp.j) {
    op[0] = cconj(sp.v0); op[3] = zero;
  } else if (sp.kind == MPO_ADJ_B && k == sp.j) {  // v0 |0><0|
    op[0] = sp.v0; op[3] = zero;
  }
  if (k == sp.lo) {
    cplx<T> w = br == 0 ? sp.w0 : sp.w1;
    for (int i = 0; i < 4; ++i) op[i] = cmul(w, op[i]);
  }
}

// ---------------------------------------------------------------------------
// Shared-memory layout of the round kernel.
template <typename T>
struct Smem {
  uint64_t *tx, *tz, *ppx, *ppz;
  uint8_t *tm;
  int *chi, *perm, *misc;
  int64_t *off;  // span offsets: Ap stack [n+2], G stack [n+2]
  int64_t *goff;
  double *red;
  double *dmisc;
  cplx<T> *tile;
  cplx<T> *jbuf, *uvec;
  int *rdim;
  T *lam;
  MpoSpec<T> *spec;
};

template <typename T>
__host__ __device__ size_t smem_bytes(int n, int W, int svd_elems) {
  size_t b = 0;
  auto add = [&](size_t bytes) { b += (bytes + 15) & ~size_t(15); };
  add(sizeof(uint64_t) * 2 * n * W);  // tx
  add(sizeof(uint64_t) * 2 * n * W);  // tz
  add(sizeof(uint64_t) * W);          // ppx
  add(sizeof(uint64_t) * W);          // ppz
  add(2 * n);                         // tm
  add(sizeof(int) * (n + 2));         // chi
  add(sizeof(int) * 512);             // perm
  add(sizeof(int) * 16);              // misc
  add(sizeof(int64_t) * (n + 2));     // off
  add(sizeof(int64_t) * (n + 2));     // goff
  add(sizeof(double) * kThreads);     // red
  add(sizeof(double) * 24);           // dmisc
  add(sizeof(cplx<T>) * kBK * (kBM + kPad + kBN + kPad));  // tile
  add(sizeof(cplx<T>) * svd_elems);  // jbuf
  add(sizeof(cplx<T>) * kMaxVec);     // uvec
  add(sizeof(int) * (n + 2));         // rdim
  add(sizeof(T) * kLamElems);         // lam (also the register-visit reductions)
  add(sizeof(MpoSpec<T>));
  return b;
}

template <typename T>
static __device__ Smem<T> carve(char *base, int n, int W, int svd_elems) {
  Smem<T> s;
  size_t b = 0;
  auto take = [&](size_t bytes) {
    char *p = base + b;
    b += (bytes + 15) & ~size_t(15);
    return p;
  };
  s.tx = reinterpret_cast<uint64_t *>(take(sizeof(uint64_t) * 2 * n * W));
  s.tz = reinterpret_cast<uint64_t *>(take(sizeof(uint64_t) * 2 * n * W));
  s.ppx = reinterpret_cast<uint64_t *>(take(sizeof(uint64_t) * W));
  s.ppz = reinterpret_cast<uint64_t *>(take(sizeof(uint64_t) * W));
  s.tm = reinterpret_cast<uint8_t *>(take(2 * n));
  s.chi = reinterpret_cast<int *>(take(sizeof(int) * (n + 2)));
  s.perm = reinterpret_cast<int *>(take(sizeof(int) * 512));
  s.misc = reinterpret_cast<int *>(take(sizeof(int) * 16));
  s.off = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * (n + 2)));
  s.goff = reinterpret_cast<int64_t *>(take(sizeof(int64_t) * (n + 2)));
  s.red = reinterpret_cast<double *>(take(sizeof(double) * kThreads));
  s.dmisc = reinterpret_cast<double *>(take(sizeof(double) * 24));
  s.tile = reinterpret_cast<cplx<T> *>(take(sizeof(cplx<T>) * kBK * (kBM + kPad + kBN + kPad)));
  s.jbuf = reinterpret_cast<cplx<T> *>(take(sizeof(cplx<T>) * svd_elems));
  s.uvec = reinterpret_cast<cplx<T> *>(take(sizeof(cplx<T>) * kMaxVec));
  s.rdim = reinterpret_cast<int *>(take(sizeof(int) * (n + 2)));
  s.lam = reinterpret_cast<T *>(take(sizeof(T) * kLamElems));
  s.spec = reinterpret_cast<MpoSpec<T> *>(take(sizeof(MpoSpec<T>)));
  return s;
}

// misc slots
// (M_JFLAG + 1 holds the blocked Jacobi's sweep flag; M_TICKET the shot taken from the queue)
enum { M_LO = 0, M_HI, M_A, M_B, M_CENTER, M_FAIL, M_KEEP, M_MAXCHI, M_CASEB, M_J, M_BIT, M_LIDX, M_OUTCOME, M_JFLAG,
       M_TICKET = 15 };
// dmisc slots
enum { D_DISC = 0, D_LOGP, D_E, D_NORM, D_FLOPS = 8, D_PROF = 8 };  // D_PROF + 1 + ProfSlot

// Adds the cycles since `t` to a phase slot and restarts `t` (thread 0 only;
// callers sit just after a CTA barrier so the CTA is in step).
__device__ __forceinline__ void prof_mark(double *dmisc, int slot, long long &t) {
  if (threadIdx.x == 0) {
    const long long now = clock64();
    dmisc[D_PROF + 1 + slot] += static_cast<double>(now - t);
    t = now;
  }
}

// Per-CTA scratch partition (complex elements).
template <typename T>
struct Scratch {
  cplx<T> *ap, *g, *t, *y, *h, *v, *vs, *w, *mbuf, *e, *sa, *te;
  T *lam;
};

template <typename T>
static __device__ Scratch<T> scratch_for(const EngineParams &P, int cap) {
  Scratch<T> s;
  cplx<T> *base = reinterpret_cast<cplx<T> *>(P.scratch) + static_cast<int64_t>(blockIdx.x) * P.scratch_elems;
  const int64_t c2 = static_cast<int64_t>(cap) * cap;
  s.ap = base;
  s.g = s.ap + P.ap_elems;
  s.t = s.g + P.g_elems;
  s.y = s.t + 8 * c2;
  s.h = s.y + 4 * c2;
  s.v = s.h + 4 * c2;
  s.vs = s.v + 4 * c2;
  s.w = s.vs + 4 * c2;
  s.mbuf = s.w + 2 * c2;
  s.e = s.mbuf + 4 * c2;
  s.sa = s.e + c2;
  s.te = s.sa + 2 * c2;
  s.lam = reinterpret_cast<T *>(s.te + 2 * c2);
  return s;
}

// Algorithmic FLOP counts (real flops of the textbook algorithm, complex = 4
// real multiply-adds per multiply-add): a GEMM is 8 M N K, a Householder R
// factor of an m x n matrix 4 (2 m n^2 - 2 n^3 / 3) with m >= n, the
// singular values and the vectors of the smaller side of an m x n matrix
// 4 (4 m n^2 + 8 n^3) with m >= n (roles swapped otherwise in both).
static __device__ __forceinline__ double gemm_flops(int M, int N, int K) { return 8.0 * M * N * K; }
static __device__ __forceinline__ double qr_flops(int m, int n) {
  double a = m >= n ? m : n, b = m >= n ? n : m;
  return 4.0 * (2.0 * a * b * b - 2.0 * b * b * b / 3.0);
}
static __device__ __forceinline__ double svd_flops(int m, int n) {
  double a = m >= n ? m : n, b = m >= n ? n : m;
  return 4.0 * (4.0 * a * b * b + 8.0 * b * b * b);
}

// ---------------------------------------------------------------------------
// MPS pieces (CTA-wide).
template <typename T>
__device__ __forceinline__ cplx<T> *site_ptr(const EngineParams &P, int64_t shot, int k) {
  return reinterpret_cast<cplx<T> *>(P.mps) + shot * P.slab_elems + P.site_off[k];
}

// out = branch-summed MPO tensor of site k (see header comment): left bond
// doubled when dl, right bond doubled when dr; the (alpha, l) index is
// alpha * chl + l.
template <typename T>
static __device__ void materialize(const MpoSpec<T> &sp, const uint64_t *ppx, const uint64_t *ppz, int k,
                            const cplx<T> *A, int chl, int chr, bool dl, bool dr, cplx<T> *out) {
  if (sp.kind == MPO_PROJ_Z) {
    // (I + s Z_S)/2 written without its two cancelling branches: the bond
    // index carries the parity of the S bits to the left, a site in S adds
    // its own bit, and the last site keeps only the target parity.  All
    // entries are 0 or 1, so a small Born probability is not the difference
    // of two numbers of order one.
    const bool in_s = (ppz[k >> 6] >> (k & 63)) & 1;
    const int Dl = dl ? 2 * chl : chl, Dr = dr ? 2 * chr : chr;
    const int64_t total = static_cast<int64_t>(Dl) * 2 * Dr;
    for (int64_t e = tid(); e < total; e += kThreads) {
      const int R = static_cast<int>(e % Dr);
      const int sb = static_cast<int>((e / Dr) % 2);
      const int L = static_cast<int>(e / (2 * Dr));
      const int al = dl ? L / chl : 0, l = dl ? L % chl : L;
      const int be = dr ? R / chr : sp.par, r = dr ? R % chr : R;
      const bool keep = in_s ? ((al ^ sb) == be) : (al == be);
      out[e] = keep ? A[(static_cast<int64_t>(l) * 2 + sb) * chr + r] : cmake<T>(0, 0);
    }
    return;
  }
  cplx<T> op0[4], op1[4];
  site_op(sp, ppx, ppz, k, 0, op0);
  site_op(sp, ppx, ppz, k, 1, op1);
  const int Dl = dl ? 2 * chl : chl, Dr = dr ? 2 * chr : chr;
  const int64_t total = static_cast<int64_t>(Dl) * 2 * Dr;
  for (int64_t e = tid(); e < total; e += kThreads) {
    int R = static_cast<int>(e % Dr);
    int s = static_cast<int>((e / Dr) % 2);
    int L = static_cast<int>(e / (2 * Dr));
    int al = dl ? L / chl : -1, l = dl ? L % chl : L;
    int be = dr ? R / chr : -1, r = dr ? R % chr : R;
    cplx<T> val = cmake<T>(0, 0);
    if (!(dl && dr && al != be)) {
      int br = dl ? al : be;
      cplx<T> a0 = A[(static_cast<int64_t>(l) * 2 + 0) * chr + r];
      cplx<T> a1 = A[(static_cast<int64_t>(l) * 2 + 1) * chr + r];
      if (br < 0) {
        cfma(val, cadd(op0[s * 2 + 0], op1[s * 2 + 0]), a0);
        cfma(val, cadd(op0[s * 2 + 1], op1[s * 2 + 1]), a1);
      } else {
        const cplx<T> *op = br == 0 ? op0 : op1;
        cfma(val, op[s * 2 + 0], a0);
        cfma(val, op[s * 2 + 1], a1);
      }
    }
    out[e] = val;
  }
}

// Keep count at one bond from eigenvalues sorted in decreasing order.
template <typename T>
static __device__ int keep_count(const T *lam_sorted, int n, int cap, double cutoff, double delta) {
  double s1 = sqrt(fmax(static_cast<double>(lam_sorted[0]), 0.0));
  if (!(s1 > 0.0)) return 1;
  int k = 0;
  for (int i = 0; i < n; ++i)
    if (sqrt(fmax(static_cast<double>(lam_sorted[i]), 0.0)) > cutoff * s1) ++k;
  if (k < 1) k = 1;
  if (k > cap) {
    double thr = sqrt(fmax(static_cast<double>(lam_sorted[cap]), 0.0)) + delta * s1;
    int kk = 0;
    for (int i = 0; i < cap; ++i)
      if (sqrt(fmax(static_cast<double>(lam_sorted[i]), 0.0)) > thr) ++kk;
    k = kk < 1 ? 1 : kk;
  }
  return k;
}

// Exact gauge steps (no truncation) moving the orthogonality centre of a
// shot's MPS from its current site to `target`, so that the sites left of an
// operator's support are left-canonical and those right of it
// right-canonical before the operator is applied (Sec. IV B).
//   Right across site k: A_k as a (2 chi_k) x chi_{k+1} matrix = Q R
//   (Householder); site k becomes Q (bond k+1 becomes min(2 chi_k,
//   chi_{k+1})) and A_{k+1} <- R A_{k+1}.
//   Left across site k: A_k^dag as a (2 chi_{k+1}) x chi_k matrix = Q R;
//   site k becomes Q^dag and A_{k-1} <- A_{k-1} R^dag.
template <typename T>
static __device__ void mps_move_center(const EngineParams &P, const Smem<T> &S, int64_t shot, const Scratch<T> &X,
                                int target) {
  int *chi = S.chi;
  const cplx<T> one = cmake<T>(1, 0), zero = cmake<T>(0, 0);
  int c = S.misc[M_CENTER];
  while (c < target) {
    const int l = chi[c], r = chi[c + 1], r2 = chi[c + 2];
    const int m = 2 * l, steps = min(m, r);
    if (m > kMaxVec) {
      if (tid() == 0) S.misc[M_FAIL] = STN_EOVERFLOW;
      __syncthreads();
      return;
    }
    cplx<T> *A = site_ptr<T>(P, shot, c), *Bn = site_ptr<T>(P, shot, c + 1);
    for (int e = tid(); e < m * r; e += kThreads) X.t[e] = A[e];
    __syncthreads();
    qr_r_inplace<T>(m, r, X.t, r, S.jbuf, P.svd_elems, S.red, S.dmisc + 4, X.h);
    form_q<T>(m, steps, X.h, X.y, S.jbuf, P.svd_elems);
    cgemm<T, 0, 0>(steps, 2 * r2, r, one, X.t, r, Bn, 2 * r2, zero, X.w, 2 * r2, S.tile);
    for (int e = tid(); e < m * steps; e += kThreads) A[e] = X.y[e];
    for (int e = tid(); e < steps * 2 * r2; e += kThreads) Bn[e] = X.w[e];
    if (tid() == 0) {
      chi[c + 1] = steps;
      S.dmisc[D_FLOPS] += 2.0 * qr_flops(m, r) + gemm_flops(steps, 2 * r2, r);
      S.dmisc[D_PROF + 1 + PROF_NGAUGE] += 1.0;
    }
    __syncthreads();
    ++c;
  }
  while (c > target) {
    const int l = chi[c], r = chi[c + 1], ll = chi[c - 1];
    const int m = 2 * r, steps = min(m, l);
    if (m > kMaxVec) {
      if (tid() == 0) S.misc[M_FAIL] = STN_EOVERFLOW;
      __syncthreads();
      return;
    }
    cplx<T> *A = site_ptr<T>(P, shot, c), *Am = site_ptr<T>(P, shot, c - 1);
    for (int e = tid(); e < m * l; e += kThreads) {
      const int j = e / l, i = e % l;  // X.t[j][i] = conj(A[i][j]), A as l x 2r
      X.t[e] = cconj(A[static_cast<int64_t>(i) * m + j]);
    }
    __syncthreads();
    qr_r_inplace<T>(m, l, X.t, l, S.jbuf, P.svd_elems, S.red, S.dmisc + 4, X.h);
    form_q<T>(m, steps, X.h, X.y, S.jbuf, P.svd_elems);
    cgemm<T, 0, 1>(2 * ll, steps, l, one, Am, l, X.t, l, zero, X.w, steps, S.tile);
    for (int e = tid(); e < steps * m; e += kThreads) {
      const int k = e / m, j = e % m;
      A[e] = cconj(X.y[static_cast<int64_t>(j) * steps + k]);
    }
    for (int e = tid(); e < 2 * ll * steps; e += kThreads) Am[e] = X.w[e];
    if (tid() == 0) {
      chi[c] = steps;
      S.dmisc[D_FLOPS] += 2.0 * qr_flops(m, l) + gemm_flops(2 * ll, steps, l);
      S.dmisc[D_PROF + 1 + PROF_NGAUGE] += 1.0;
    }
    __syncthreads();
    --c;
  }
  if (tid() == 0) S.misc[M_CENTER] = target;
  __syncthreads();
}

// Two phases of applying the two-branch MPO `spec` on [lo, hi] and
// recompressing sites [a, b] (a <= lo <= hi <= b, orthogonality centre inside
// [a, b]).
//
// mps_prepare builds the MPO tensors and runs the left sweep (no truncation
// yet) and returns the squared norm of the new, untruncated state: for a
// measurement projector this is the Born probability of the branch, obtained
// from R factors whose small entries carry absolute (not relative) rounding,
// so a small probability keeps its relative accuracy (about eps / sqrt(p)).
// mps_finish then runs the truncating right sweep; the centre ends at a and the
// state is renormalised.
template <typename T>
static __device__ double mps_prepare(const EngineParams &P, const Smem<T> &S, int64_t shot,
                              const Scratch<T> &X, int a, int b) {
  const MpoSpec<T> &sp = *S.spec;
  int *chi = S.chi;
  if (a == b) {
    cplx<T> *A = site_ptr<T>(P, shot, a);
    materialize(sp, S.ppx, S.ppz, a, A, chi[a], chi[a + 1], false, false, X.t);
    __syncthreads();
    const int64_t tot = static_cast<int64_t>(chi[a]) * 2 * chi[a + 1];
    double nrm = 0;
    for (int64_t e = tid(); e < tot; e += kThreads) nrm += cabs2d(X.t[e]);
    return block_sum(nrm, S.red);
  }
  // doubled bond dimensions D[k] for bonds a..b+1
  auto Dbond = [&](int k) { return (k > sp.lo && k <= sp.hi) ? 2 * chi[k] : chi[k]; };
  if (tid() == 0) {
    int64_t o = 0;
    for (int k = a; k <= b; ++k) {
      S.off[k - a] = o;
      o += static_cast<int64_t>(Dbond(k)) * 2 * Dbond(k + 1);
    }
    S.off[b - a + 1] = o;
    int64_t g = 0;
    for (int k = a + 1; k <= b; ++k) {
      S.goff[k - a] = g;
      g += static_cast<int64_t>(Dbond(k)) * Dbond(k);
    }
    S.goff[b - a + 1] = g;
    if (o > P.ap_elems || g > P.g_elems) S.misc[M_FAIL] = STN_EOVERFLOW;
  }
  __syncthreads();
  if (S.misc[M_FAIL]) return 0.0;
  for (int k = a; k <= b; ++k) {
    bool in = k >= sp.lo && k <= sp.hi;
    bool dl = in && k > sp.lo, dr = in && k < sp.hi;
    cplx<T> *A = site_ptr<T>(P, shot, k);
    cplx<T> *out = X.ap + S.off[k - a];
    if (in) {
      materialize(sp, S.ppx, S.ppz, k, A, chi[k], chi[k + 1], dl, dr, out);
    } else {
      const int64_t tot = static_cast<int64_t>(chi[k]) * 2 * chi[k + 1];
      for (int64_t e = tid(); e < tot; e += kThreads) out[e] = A[e];
    }
  }
  __syncthreads();
  const cplx<T> one = cmake<T>(1, 0), zero = cmake<T>(0, 0);
  const int cap = P.chi_cap;
  (void)cap;
  // left sweep: R factor of the left part through site k, for k = a..b-1
  // (R at bond a is the identity: sites left of a are left-canonical).
  for (int k = a; k < b; ++k) {
    const int Dl = Dbond(k), Dr = Dbond(k + 1);
    const cplx<T> *Ak = X.ap + S.off[k - a];
    int m;
    if (k == a) {
      m = 2 * Dl;
      const int64_t tot = static_cast<int64_t>(m) * Dr;
      for (int64_t e = tid(); e < tot; e += kThreads) X.t[e] = Ak[e];
      __syncthreads();
    } else {
      const int r = S.rdim[k - a];
      const cplx<T> *Rk = X.g + S.goff[k - a];
      cgemm<T, 0, 0>(r, 2 * Dr, Dl, one, Rk, Dl, Ak, 2 * Dr, zero, X.t, 2 * Dr, S.tile);
      if (tid() == 0) S.dmisc[D_FLOPS] += gemm_flops(r, 2 * Dr, Dl);
      m = 2 * r;
    }
    if (m > kMaxVec) {
      if (tid() == 0) S.misc[M_FAIL] = STN_EOVERFLOW;
      __syncthreads();
      return 0.0;
    }
    qr_r_inplace<T>(m, Dr, X.t, Dr, S.jbuf, P.svd_elems, S.red, S.dmisc + 4);
    if (tid() == 0) S.dmisc[D_FLOPS] += qr_flops(m, Dr);
    const int rn = min(m, Dr);
    cplx<T> *Rout = X.g + S.goff[k + 1 - a];
    for (int e = tid(); e < rn * Dr; e += kThreads) Rout[e] = X.t[e];
    if (tid() == 0) S.rdim[k + 1 - a] = rn;
    __syncthreads();
  }
  // squared norm: || R_b A'_b ||_F^2 (the right part beyond b is right-canonical)
  {
    const int Dl = Dbond(b), n2 = 2 * Dbond(b + 1), r = S.rdim[b - a];
    cgemm<T, 0, 0>(r, n2, Dl, one, X.g + S.goff[b - a], Dl, X.ap + S.off[b - a], n2, zero, X.y, n2, S.tile);
    double nrm = 0;
    for (int e = tid(); e < r * n2; e += kThreads) nrm += cabs2d(X.y[e]);
    return block_sum(nrm, S.red);
  }
}

template <typename T>
static __device__ void mps_finish(const EngineParams &P, const Smem<T> &S, int64_t shot, const Scratch<T> &X,
                           int a, int b) {
  const MpoSpec<T> &sp = *S.spec;
  int *chi = S.chi;
  const int cap = P.chi_cap;
  if (S.misc[M_FAIL]) return;
  if (a == b) {
    cplx<T> *A = site_ptr<T>(P, shot, a);
    const int64_t tot = static_cast<int64_t>(chi[a]) * 2 * chi[a + 1];
    double nrm = 0;
    for (int64_t e = tid(); e < tot; e += kThreads) nrm += cabs2d(X.t[e]);
    nrm = block_sum(nrm, S.red);
    T inv = static_cast<T>(nrm > 0 ? 1.0 / sqrt(nrm) : 0.0);
    for (int64_t e = tid(); e < tot; e += kThreads) A[e] = cscale(X.t[e], inv);
    if (tid() == 0) {
      if (!(nrm > 0) || !isfinite(nrm)) S.misc[M_FAIL] = STN_ENUMERIC;
      S.misc[M_CENTER] = a;
    }
    __syncthreads();
    return;
  }
  auto Dbond = [&](int k) { return (k > sp.lo && k <= sp.hi) ? 2 * chi[k] : chi[k]; };
  const cplx<T> one = cmake<T>(1, 0), zero = cmake<T>(0, 0);
  long long tp = clock64();
  // right sweep
  int kappa = Dbond(b + 1);
  const cplx<T> *M = X.ap + S.off[b - a];
  for (int k = b; k > a; --k) {
    const int Dl = Dbond(k);
    const int n2 = 2 * kappa;
    const int r = S.rdim[k - a];
    const cplx<T> *Rk = X.g + S.goff[k - a];
    // C = R_k M (r x n2), then its SVD
    cgemm<T, 0, 0>(r, n2, Dl, one, Rk, Dl, M, n2, zero, X.y, n2, S.tile);
    prof_mark(S.dmisc, PROF_RIGHT, tp);
    const bool in_smem = r * n2 + n2 * n2 <= P.svd_elems;
    cplx<T> *Cc = in_smem ? S.jbuf : X.h;
    cplx<T> *Vc = in_smem ? S.jbuf + r * n2 : X.v;
    // In the complex64 path a bond whose SVD fits shared memory in complex128
    // is decomposed in double precision: FP32 Jacobi rotations leave the small
    // singular directions with an absolute error of about sqrt(#rotations)
    // eps sigma_1, which would be dropped or kept wrongly at every sweep.
    bool svd64 = false, vec_from_columns = false;
    if constexpr (sizeof(T) == 4) svd64 = 2 * (r * n2 + n2 * n2) <= P.svd_elems;
    if (svd64) {
      cplx<double> *Cd = reinterpret_cast<cplx<double> *>(S.jbuf), *Vd = Cd + r * n2;
      double *sd = reinterpret_cast<double *>(X.te);
      for (int e = tid(); e < r * n2; e += kThreads) {
        int i = e / n2, j = e % n2;
        cplx<T> v = X.y[e];
        Cd[j * r + i] = cmake<double>(static_cast<double>(v.re), static_cast<double>(v.im));
      }
      __syncthreads();
      svd_onesided<double>(r, n2, Cd, Vd, sd, &S.misc[M_JFLAG], S.red);
      for (int e = tid(); e < n2 * n2; e += kThreads)
        X.v[e] = cmake<T>(static_cast<T>(Vd[e].re), static_cast<T>(Vd[e].im));
      for (int i = tid(); i < n2; i += kThreads) X.lam[i] = static_cast<T>(sd[i]);
      __syncthreads();
      Vc = X.v;
    } else if (sizeof(T) == 4 && P.svd64_all) {
      // Complex64 contractions with every SVD in double precision: the large
      // path (Householder R factor, Jacobi on R^dag) on a complex128 copy of
      // C in the scratch areas h and v (contiguous, 4 c^2 complex128), with
      // the shared buffer as complex128 staging; the rotated columns come back
      // in single precision.
      if (r > kMaxVec) {
        if (tid() == 0) S.misc[M_FAIL] = STN_EOVERFLOW;
        __syncthreads();
        return;
      }
      cplx<double> *Cd = reinterpret_cast<cplx<double> *>(X.h);
      cplx<double> *jd = reinterpret_cast<cplx<double> *>(S.jbuf);
      double *sd = reinterpret_cast<double *>(X.te);
      for (int e = tid(); e < r * n2; e += kThreads)
        Cd[e] = cmake<double>(static_cast<double>(X.y[e].re), static_cast<double>(X.y[e].im));
      __syncthreads();
      const long long tqr = clock64();
      qr_r_inplace<double>(r, n2, Cd, n2, jd, P.svd_elems / 2, S.red, S.dmisc + 4);
      if (tid() == 0) S.dmisc[D_PROF + 1 + PROF_SVD_QR] += static_cast<double>(clock64() - tqr);
      const int kx = min(r, n2);
      for (int e = tid(); e < n2 * kx; e += kThreads) Cd[e] = cconj(Cd[e]);
      __syncthreads();
      const long long tj = clock64();
      const int sweeps = svd_onesided_blocked<double>(n2, kx, Cd, nullptr, sd, &S.misc[M_JFLAG], S.red, jd,
                                                      P.svd_elems / 2);
      if (tid() == 0) {
        S.dmisc[D_PROF + 1 + PROF_JSWEEPS] += sweeps;
        S.dmisc[D_PROF + 1 + PROF_JROWS] += n2;
        S.dmisc[D_PROF + 1 + PROF_JCOLS] += kx;
        if (n2 <= kThreads / 2) S.dmisc[D_PROF + 1 + PROF_JAC_ROWS256] += static_cast<double>(clock64() - tj);
      }
      for (int e = tid(); e < n2 * kx; e += kThreads)
        X.y[e] = cmake<T>(static_cast<T>(Cd[e].re), static_cast<T>(Cd[e].im));
      for (int i = tid(); i < n2; i += kThreads) X.lam[i] = i < kx ? static_cast<T>(sd[i]) : T(0);
      __syncthreads();
      Vc = X.y;
      vec_from_columns = true;
    } else if (in_smem) {
      for (int e = tid(); e < r * n2; e += kThreads) {
        int i = e / n2, j = e % n2;
        Cc[j * r + i] = X.y[e];
      }
      __syncthreads();
      svd_onesided<T>(r, n2, Cc, Vc, X.lam, &S.misc[M_JFLAG], S.red);
    } else {
      // Large bond: C = Q1 R1 (Householder), then one-sided Jacobi on
      // X = R1^dag (n2 x kx), whose columns converge in a few sweeps because
      // R1 is already nearly diagonal.  X V_x = U_x Sigma gives
      // R1 = V_x Sigma U_x^dag, so the right singular vectors of C are the
      // normalised columns of the rotated X and no rotation is accumulated.
      // Rows of R1 (row-major, ld n2) are the conjugated columns of X
      // (column-major, ld n2) in place.
      if (r > kMaxVec) {
        if (tid() == 0) S.misc[M_FAIL] = STN_EOVERFLOW;
        __syncthreads();
        return;
      }
      const long long tqr = clock64();
      qr_r_inplace<T>(r, n2, X.y, n2, S.jbuf, P.svd_elems, S.red, S.dmisc + 4);
      if (tid() == 0) S.dmisc[D_PROF + 1 + PROF_SVD_QR] += static_cast<double>(clock64() - tqr);
      const int kx = min(r, n2);
      // complex64 with more than one block of 16 columns: blocked Jacobi
      // with register-resident block pairs, X in global scratch (L2)
      const bool regs = sizeof(T) == 4 && kx > 16 && n2 <= kThreads;
      const bool x_smem = !regs && n2 * kx <= P.svd_elems;
      cplx<T> *Xc = x_smem ? S.jbuf : X.y;
      for (int e = tid(); e < n2 * kx; e += kThreads) Xc[e] = cconj(X.y[e]);
      __syncthreads();
      const long long tj = clock64();
      const int sweeps =
          x_smem ? svd_onesided<T>(n2, kx, Xc, nullptr, X.lam, &S.misc[M_JFLAG], S.red)
                 : svd_onesided_blocked<T>(n2, kx, Xc, nullptr, X.lam, &S.misc[M_JFLAG], S.red, S.jbuf,
                                           P.svd_elems, regs ? reinterpret_cast<float *>(S.lam) : nullptr);
      if (tid() == 0) {
        S.dmisc[D_PROF + 1 + PROF_JSWEEPS] += sweeps;
        S.dmisc[D_PROF + 1 + PROF_JROWS] += n2;
        S.dmisc[D_PROF + 1 + PROF_JCOLS] += kx;
        if (n2 <= kThreads / 2) S.dmisc[D_PROF + 1 + PROF_JAC_ROWS256] += static_cast<double>(clock64() - tj);
      }
      for (int i = kx + tid(); i < n2; i += kThreads) X.lam[i] = T(0);
      __syncthreads();
      Vc = Xc;
      vec_from_columns = true;
    }
    __syncthreads();
    if (tid() == 0 && !vec_from_columns) S.dmisc[D_PROF + 1 + PROF_SVD_SMALL] += static_cast<double>(clock64() - tp);
    prof_mark(S.dmisc, PROF_SVD, tp);
    if (tid() == 0) {
      S.dmisc[D_FLOPS] += gemm_flops(r, n2, Dl) + svd_flops(r, n2);
      S.dmisc[D_PROF + 1 + (vec_from_columns ? PROF_NSVD_LARGE : PROF_NSVD_SMALL)] += 1.0;
    }
    for (int i = tid(); i < n2; i += kThreads) {
      if (!isfinite(static_cast<double>(X.lam[i]))) {
        S.misc[M_FAIL] = STN_ENUMERIC;
        X.lam[i] = T(0);
      }
    }
    __syncthreads();
    if (S.misc[M_FAIL]) return;
    sort_desc<T>(n2, X.lam, S.perm);
    for (int i = tid(); i < n2; i += kThreads) S.lam[i] = X.lam[S.perm[i]];
    __syncthreads();
    if (tid() == 0) {
      int kmax = min(cap, P.chimax[k]);
      int keep = keep_count<T>(S.lam, n2, kmax, P.cutoff, P.delta);
      if (keep > kmax) keep = kmax;
      double tot = 0, drop = 0;
      for (int i = 0; i < n2; ++i) {
        double l = fmax(static_cast<double>(S.lam[i]), 0.0);
        tot += l;
        if (i >= keep) drop += l;
      }
      if (tot > 0) S.dmisc[D_DISC] += drop / tot;
      S.misc[M_KEEP] = keep;
    }
    __syncthreads();
    const int keep = S.misc[M_KEEP];
    // sorted, kept right singular vectors: Vs[:, c] = V[:, perm[c]], c < keep
    // (or the rotated column of X over its norm)
    for (int e = tid(); e < n2 * keep; e += kThreads) {
      int i = e / keep, c = e % keep;
      cplx<T> v = Vc[static_cast<int64_t>(S.perm[c]) * n2 + i];
      if (vec_from_columns) {
        T l = S.lam[c];
        v = l > T(0) ? cscale(v, T(1) / sqrt(l)) : cmake<T>(i == c ? T(1) : T(0), 0);
      }
      X.vs[i * keep + c] = v;
    }
    __syncthreads();
    reorthonormalize<T>(n2, keep, X.vs, X.e, X.y, S.tile);
    // new right-canonical site k: B[c][s][r] = conj(Vs[(s*kappa + r)][c])
    cplx<T> *Bk = site_ptr<T>(P, shot, k);
    for (int e = tid(); e < keep * n2; e += kThreads) {
      int c = e / n2, sr = e % n2;
      Bk[e] = cconj(X.vs[sr * keep + c]);
    }
    // W = M Vs (Dl x keep)
    cgemm<T, 0, 0>(Dl, keep, n2, one, M, n2, X.vs, keep, zero, X.w, keep, S.tile);
    // M_{k-1} = A'_{k-1} (left reshape 2D_{k-1} x Dl) W
    const int Dll = Dbond(k - 1);
    const cplx<T> *Akm1 = X.ap + S.off[k - 1 - a];
    cgemm<T, 0, 0>(2 * Dll, keep, Dl, one, Akm1, Dl, X.w, keep, zero, X.mbuf, keep, S.tile);
    if (tid() == 0) {
      chi[k] = keep;
      S.dmisc[D_FLOPS] += gemm_flops(Dl, keep, n2) + gemm_flops(2 * Dll, keep, Dl);
    }
    __syncthreads();
    M = X.mbuf;
    kappa = keep;
  }
  prof_mark(S.dmisc, PROF_RIGHT, tp);
  // centre site a = M (chi[a] x 2 x kappa), renormalised
  cplx<T> *Aa = site_ptr<T>(P, shot, a);
  const int64_t tot = static_cast<int64_t>(chi[a]) * 2 * kappa;
  double nrm = 0;
  for (int64_t e = tid(); e < tot; e += kThreads) nrm += cabs2d(M[e]);
  nrm = block_sum(nrm, S.red);
  T inv = static_cast<T>(nrm > 0 ? 1.0 / sqrt(nrm) : 0.0);
  for (int64_t e = tid(); e < tot; e += kThreads) Aa[e] = cscale(M[e], inv);
  if (tid() == 0) {
    if (!(nrm > 0) || !isfinite(nrm)) S.misc[M_FAIL] = STN_ENUMERIC;
    S.misc[M_CENTER] = a;
    int mx = S.misc[M_MAXCHI];
    for (int k = a + 1; k <= b; ++k) mx = max(mx, chi[k]);
    S.misc[M_MAXCHI] = mx;
  }
  __syncthreads();
}

// <phi| i^m X^x Z^z |phi> over sites [a, b] (centre inside, so the rest of
// the chain contracts to the identity).  Returns the real part.
template <typename T>
static __device__ double mps_expect(const EngineParams &P, const Smem<T> &S, int64_t shot,
                             const Scratch<T> &X, int a, int b, int m) {
  const int *chi = S.chi;
  const cplx<T> one = cmake<T>(1, 0), zero = cmake<T>(0, 0);
  MpoSpec<T> sp;
  sp.kind = MPO_ROT; sp.lo = -1; sp.hi = -1; sp.j = -1;
  sp.w0 = one; sp.w1 = one; sp.v0 = zero; sp.v1 = zero;
  for (int k = a; k <= b; ++k) {
    const cplx<T> *A = site_ptr<T>(P, shot, k);
    const int cl = chi[k], cr = chi[k + 1];
    // SA = (X^x Z^z)_k A_k
    cplx<T> op[4];
    site_op(sp, S.ppx, S.ppz, k, 1, op);
    const int64_t tot = static_cast<int64_t>(cl) * 2 * cr;
    for (int64_t e = tid(); e < tot; e += kThreads) {
      int r = static_cast<int>(e % cr), s = static_cast<int>((e / cr) % 2);
      int64_t l = e / (2 * cr);
      cplx<T> v = cmake<T>(0, 0);
      cfma(v, op[s * 2 + 0], A[(l * 2 + 0) * cr + r]);
      cfma(v, op[s * 2 + 1], A[(l * 2 + 1) * cr + r]);
      X.sa[e] = v;
    }
    __syncthreads();
    if (k == a) {
      cgemm<T, 1, 0>(cr, cr, 2 * cl, one, A, cr, X.sa, cr, zero, X.e, cr, S.tile);
      if (tid() == 0) S.dmisc[D_FLOPS] += gemm_flops(cr, cr, 2 * cl);
    } else {
      cgemm<T, 0, 0>(cl, 2 * cr, cl, one, X.e, cl, X.sa, 2 * cr, zero, X.te, 2 * cr, S.tile);
      cgemm<T, 1, 0>(cr, cr, 2 * cl, one, A, cr, X.te, cr, zero, X.e, cr, S.tile);
      if (tid() == 0) S.dmisc[D_FLOPS] += gemm_flops(cl, 2 * cr, cl) + gemm_flops(cr, cr, 2 * cl);
    }
  }
  const int cb = chi[b + 1];
  double re = 0, im = 0;
  for (int i = tid(); i < cb; i += kThreads) {
    re += static_cast<double>(X.e[i * cb + i].re);
    im += static_cast<double>(X.e[i * cb + i].im);
  }
  re = block_sum(re, S.red);
  im = block_sum(im, S.red);
  // multiply by i^m, keep the real part
  switch (m & 3) {
    case 0: return re;
    case 1: return -im;
    case 2: return -re;
    default: return im;
  }
}

// ---------------------------------------------------------------------------
// Tableau helpers (shared memory, one thread unless noted).
static __device__ __forceinline__ int popc64(uint64_t v) { return __popcll(v); }

// row r <- row r * row s (Pauli product with the exact phase)
static __device__ void row_mul(uint64_t *tx, uint64_t *tz, uint8_t *tm, int W, int r, int s) {
  int sw = 0;
  for (int w = 0; w < W; ++w) {
    sw += popc64(tz[r * W + w] & tx[s * W + w]);
    tx[r * W + w] ^= tx[s * W + w];
    tz[r * W + w] ^= tz[s * W + w];
  }
  tm[r] = static_cast<uint8_t>((tm[r] + tm[s] + 2 * sw) & 3);
}

// rows of X errors anticommute with Z_q, and vice versa
static __device__ void pauli_left(uint8_t *tm, int n, int q, int letter /*1 X, 2 Y, 3 Z*/) {
  if (letter == 1 || letter == 2) tm[n + q] = static_cast<uint8_t>((tm[n + q] + 2) & 3);
  if (letter == 3 || letter == 2) tm[q] = static_cast<uint8_t>((tm[q] + 2) & 3);
}

// P' = row r1 * row r2 (r2 < 0: just row r1) into ppx/ppz, phase returned
static __device__ int conj_rows(const uint64_t *tx, const uint64_t *tz, const uint8_t *tm, int W, int r1,
                         int r2, uint64_t *ppx, uint64_t *ppz) {
  int m = tm[r1];
  int sw = 0;
  for (int w = 0; w < W; ++w) {
    ppx[w] = tx[r1 * W + w];
    ppz[w] = tz[r1 * W + w];
    if (r2 >= 0) {
      sw += popc64(ppz[w] & tx[r2 * W + w]);
      ppx[w] ^= tx[r2 * W + w];
      ppz[w] ^= tz[r2 * W + w];
    }
  }
  if (r2 >= 0) m += tm[r2] + 2 * sw;
  return m & 3;
}

// Single-qubit Clifford L applied to the site-j letter of every row:
// R -> L R L^dag, for the four L that take the measured eigenvector to |0>:
// index 0: X,+1 (H)  1: X,-1 (X H)  2: Y,+1 (H S^dag)  3: Y,-1 (X H S^dag).
// Table: [L][xz] -> (x', z', dm) with xz = 2x + z.
__constant__ uint8_t kLTable[4][4][3] = {
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 0}, {1, 1, 2}},
    {{0, 0, 0}, {1, 0, 0}, {0, 1, 2}, {1, 1, 0}},
    {{0, 0, 0}, {1, 0, 0}, {1, 1, 1}, {0, 1, 3}},
    {{0, 0, 0}, {1, 0, 0}, {1, 1, 3}, {0, 1, 1}},
};

// C <- C U L^dag for U = prod_{k != j} controlled-P'_k (control j): every row
// R -> L (U R U) L^dag, with U R U = R Z_j^a (x_j(R) = 0) or
// (-1)^a R Z_j^a Q (x_j(R) = 1), a = [R anticommutes with Q],
// Q = prod_{k != j} P'_k.  CTA-wide over rows.
static __device__ void tableau_caseB(uint64_t *tx, uint64_t *tz, uint8_t *tm, int n, int W,
                              const uint64_t *ppx, const uint64_t *ppz, int j, int lidx) {
  const int jw = j >> 6;
  const uint64_t jb = 1ull << (j & 63);
  for (int r = tid(); r < 2 * n; r += kThreads) {
    int an = 0, mq = 0;
    for (int w = 0; w < W; ++w) {
      uint64_t xq = ppx[w] & (w == jw ? ~jb : ~0ull);
      uint64_t zq = ppz[w] & (w == jw ? ~jb : ~0ull);
      an += popc64((tx[r * W + w] & zq) ^ (tz[r * W + w] & xq));
      mq += popc64(xq & zq);
    }
    an &= 1;
    const bool xj = (tx[r * W + jw] & jb) != 0;
    int m = tm[r];
    if (an) tz[r * W + jw] ^= jb;
    if (xj) {
      if (an) m += 2;
      int sw = 0;
      for (int w = 0; w < W; ++w) {
        uint64_t xq = ppx[w] & (w == jw ? ~jb : ~0ull);
        uint64_t zq = ppz[w] & (w == jw ? ~jb : ~0ull);
        sw += popc64(tz[r * W + w] & xq);
        tx[r * W + w] ^= xq;
        tz[r * W + w] ^= zq;
      }
      m += mq + 2 * sw;
    }
    int x = (tx[r * W + jw] & jb) ? 1 : 0, z = (tz[r * W + jw] & jb) ? 1 : 0;
    const uint8_t *e = kLTable[lidx][2 * x + z];
    if (e[0]) tx[r * W + jw] |= jb; else tx[r * W + jw] &= ~jb;
    if (e[1]) tz[r * W + jw] |= jb; else tz[r * W + jw] &= ~jb;
    tm[r] = static_cast<uint8_t>((m + e[2]) & 3);
  }
  __syncthreads();
}

// Projector MPO of outcome `bit` for the measured P' (thread 0): case A
// (no X or Y in P') projects with (I + (-1)^bit P')/2; case B applies the
// controlled-Pauli product with the site-j projection onto the lambda
// eigenvector, lambda = (-1)^bit * sign(P').
template <typename T>
static __device__ void set_meas_spec(const Smem<T> &S, int bit) {
  MpoSpec<T> &sp = *S.spec;
  const int mb = S.misc[M_BIT];
  const int m = mb & 3;
  const int neg = (mb >> 4) & 1;
  if (!S.misc[M_CASEB]) {
    // P' = i^m Z^z with m even (Hermitian, no X): keep the states whose S
    // parity makes (-1)^b i^m (-1)^parity = +1
    sp.kind = MPO_PROJ_Z;
    const int sgn = (bit ? -1 : 1) * ((m & 2) ? -1 : 1);
    sp.par = sgn > 0 ? 0 : 1;
    sp.w0 = cmake<T>(1, 0);
    sp.w1 = cmake<T>(1, 0);
  } else {
    const int jq = S.misc[M_J];
    const bool zj = (S.ppz[jq >> 6] >> (jq & 63)) & 1;
    int lam = (bit ? -1 : 1) * (neg ? -1 : 1);
    const T r2 = static_cast<T>(0.70710678118654752440);
    sp.kind = MPO_PROJ_B;
    sp.w0 = cmake<T>(1, 0);
    sp.w1 = cmake<T>(1, 0);
    sp.v0 = cmake<T>(r2, 0);
    sp.v1 = zj ? cmake<T>(0, lam > 0 ? r2 : -r2) : cmake<T>(lam > 0 ? r2 : -r2, 0);
    S.misc[M_LIDX] = (zj ? 2 : 0) + (lam < 0 ? 1 : 0);
  }
}

// ---------------------------------------------------------------------------
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) round_kernel(EngineParams P) {
  extern __shared__ __align__(16) char smem_raw[];
  const int n = P.n, W = P.W;
  Smem<T> S = carve<T>(smem_raw, n, W, P.svd_elems);
  Scratch<T> X = scratch_for<T>(P, P.work_c);
  // complex64 with use_tc (gemm_units = STN_GEMM_TENSOR): the large
  // contractions run on the tensor cores, staged in the shared SVD buffer
  // (free whenever a GEMM runs)
  bool tc_alloc = false;
  if constexpr (sizeof(T) == 4) tc_alloc = P.use_tc && static_cast<int64_t>(P.svd_elems) * 2 >= kTcStageFloats;
  if (tc_alloc) tc_setup(reinterpret_cast<float *>(S.jbuf));
  else tc_disable();
  bool tc_live = tc_alloc;  // CTA-uniform
  // With a ticket counter the CTAs take the batch's shots in order as they
  // finish (a work queue that balances uneven shots when the batch holds
  // more shots than CTAs); without one, shots are grid-strided.
  for (int64_t it = 0;; ++it) {
    int64_t shot = blockIdx.x + it * gridDim.x;
    if (P.ticket) {
      if (tid() == 0) S.misc[M_TICKET] = atomicAdd(P.ticket, 1);
      __syncthreads();
      shot = S.misc[M_TICKET];
      __syncthreads();
    }
    if (shot >= P.shots) break;
    // load the frame and the MPS bookkeeping
    for (int e = tid(); e < 2 * n * W; e += kThreads) {
      S.tx[e] = P.tab_x[shot * 2 * n * W + e];
      S.tz[e] = P.tab_z[shot * 2 * n * W + e];
    }
    for (int e = tid(); e < 2 * n; e += kThreads) S.tm[e] = P.tab_m[shot * 2 * n + e];
    for (int e = tid(); e <= n; e += kThreads) S.chi[e] = P.chi[shot * (n + 1) + e];
    if (tid() == 0) {
      S.misc[M_CENTER] = P.center[shot];
      S.misc[M_FAIL] = P.status[shot];
      S.misc[M_MAXCHI] = P.maxchi[shot];
      S.dmisc[D_DISC] = P.disc[shot];
      S.dmisc[D_LOGP] = P.logp[shot];
      S.dmisc[D_FLOPS] = 0.0;
      for (int i = 0; i < kProfSlots; ++i) S.dmisc[D_PROF + 1 + i] = 0.0;
    }
    __syncthreads();
    long long t_ops = clock64();
    const uint64_t gshot = (P.shot_offset_dev ? *P.shot_offset_dev : P.shot_offset) + static_cast<uint64_t>(shot);
    for (int oi = P.op_begin; oi < P.op_end; ++oi) {
      if (tc_live) {
        // a tensor-core wait ran out: this shot stops, the rest use the CUDA
        // cores.  Every thread reads the flag before thread 0 may clear it.
        const int tc_failed = g_tc.failed;
        __syncthreads();
        if (tc_failed) {
          if (tid() == 0) {
            S.misc[M_FAIL] = STN_ETIMEOUT;
            g_tc.failed = 0;
            g_tc.enabled = 0;
          }
          tc_live = false;
          __syncthreads();
        }
      }
      if (S.misc[M_FAIL]) break;
      const Op op = P.ops[oi];
      switch (op.kind) {
        case OP_RESET_FLIP:
          if (tid() == 0 && philox_uniform(P.seed, gshot, op.ev) < P.pR) pauli_left(S.tm, n, op.a, 1);
          break;
        case OP_H:
          if (tid() < W) {
            int w = tid();
            uint64_t t = S.tx[op.a * W + w];
            S.tx[op.a * W + w] = S.tx[(n + op.a) * W + w];
            S.tx[(n + op.a) * W + w] = t;
            t = S.tz[op.a * W + w];
            S.tz[op.a * W + w] = S.tz[(n + op.a) * W + w];
            S.tz[(n + op.a) * W + w] = t;
          }
          if (tid() == 0) {
            uint8_t t = S.tm[op.a];
            S.tm[op.a] = S.tm[n + op.a];
            S.tm[n + op.a] = t;
          }
          break;
        case OP_NOISE1:
          if (tid() == 0) {
            double u = philox_uniform(P.seed, gshot, op.ev);
            if (u < P.p1) pauli_left(S.tm, n, op.a, 1 + min(2, static_cast<int>(3.0 * u / P.p1)));
          }
          break;
        case OP_CNOT:
          if (tid() == 0) {
            row_mul(S.tx, S.tz, S.tm, W, op.a, op.b);          // X_c <- X_c X_t
            row_mul(S.tx, S.tz, S.tm, W, n + op.b, n + op.a);  // Z_t <- Z_t Z_c (rows commute)
          }
          break;
        case OP_NOISE2:
          if (tid() == 0) {
            double u = philox_uniform(P.seed, gshot, op.ev);
            if (u < P.p2) {
              int idx = min(14, static_cast<int>(15.0 * u / P.p2)) + 1;
              int lc = idx / 4, lt = idx % 4;  // 0 I, 1 X, 2 Y, 3 Z
              if (lc) pauli_left(S.tm, n, op.a, lc);
              if (lt) pauli_left(S.tm, n, op.b, lt);
            }
          }
          break;
        case OP_ROT:
        case OP_MEAS: {
          const bool meas = op.kind == OP_MEAS;
          if (tid() == 0) {
            int m;
            if (meas) m = conj_rows(S.tx, S.tz, S.tm, W, n + op.a, -1, S.ppx, S.ppz);
            else if (op.pauli == 0) m = conj_rows(S.tx, S.tz, S.tm, W, n + op.a, n + op.b, S.ppx, S.ppz);
            else m = conj_rows(S.tx, S.tz, S.tm, W, op.a, op.b, S.ppx, S.ppz);
            int lo = n, hi = -1, j = -1, xany = 0, xz = 0;
            for (int q = 0; q < n; ++q) {
              bool x = (S.ppx[q >> 6] >> (q & 63)) & 1, z = (S.ppz[q >> 6] >> (q & 63)) & 1;
              if (x || z) { lo = min(lo, q); hi = max(hi, q); }
              if (x && j < 0) j = q;
              xany |= x;
              xz += x && z;
            }
            int c = S.misc[M_CENTER];
            S.misc[M_LO] = lo;
            S.misc[M_HI] = hi;
            (void)c;
            S.misc[M_A] = lo;
            S.misc[M_B] = hi;
            S.misc[M_J] = j;
            S.misc[M_CASEB] = xany;
            S.misc[M_BIT] = m | ((((m - xz) & 3) == 2) << 4);  // phase | (sign < 0) << 4
            MpoSpec<T> &sp = *S.spec;
            sp.lo = lo; sp.hi = hi; sp.j = j;
            if (!meas) {
              double th = P.theta[op.idx];
              cplx<T> w1 = cmul(cmake<T>(0, static_cast<T>(-sin(th))), ipow<T>(m));
              sp.kind = MPO_ROT;
              sp.w0 = cmake<T>(static_cast<T>(cos(th)), 0);
              sp.w1 = w1;
            }
            if (lo > hi) S.misc[M_FAIL] = STN_ENUMERIC;  // identity Pauli cannot occur
            if (P.tape_info) {
              const int64_t t = shot * P.n_ops_total + oi;
              for (int w = 0; w < W; ++w) {
                P.tape_px[t * W + w] = S.ppx[w];
                P.tape_pz[t * W + w] = S.ppz[w];
              }
              int32_t *ti = P.tape_info + t * kTapeInts;
              ti[0] = m & 3;
              ti[1] = lo;
              ti[2] = hi;
              ti[3] = j;
            }
          }
          __syncthreads();
          if (S.misc[M_FAIL]) break;
          const int a = S.misc[M_A], b = S.misc[M_B];
          {
            // the centre moves into [a, b] by exact gauge steps; the sweep
            // then covers the operator's support only
            const int c0 = S.misc[M_CENTER];
            const int tgt = c0 < a ? a : (c0 > b ? b : c0);
            if (tgt != c0) {
              long long tg = clock64();
              mps_move_center<T>(P, S, shot, X, tgt);
              prof_mark(S.dmisc, PROF_GAUGE, tg);
            }
          }
          if (S.misc[M_FAIL]) break;
          int caseB = 0, lidx = 0, outcome = 0;
          if (meas) {
            // The Born probability of the less likely branch is the squared
            // norm of its projected state, from R factors: any deviation of
            // the sites outside [a, b] from exact isometries (rounding of the
            // gauge steps and sweeps) changes it only relatively.  The
            // expectation value only decides which branch that is.
            const int mb = S.misc[M_BIT];
            long long tq = clock64();
            const double e = mps_expect<T>(P, S, shot, X, a, b, mb & 3);
            const int small = e >= 0.0 ? 1 : 0;
            if (tid() == 0) set_meas_spec<T>(S, small);
            __syncthreads();
            prof_mark(S.dmisc, PROF_EXPECT, tq);
            const double ps = fmin(1.0, fmax(0.0, mps_prepare<T>(P, S, shot, X, a, b)));
            prof_mark(S.dmisc, PROF_LEFT, tq);
            if (tid() == 0) {
              double p0 = small == 0 ? ps : 1.0 - ps;
              double u = philox_uniform(P.seed, gshot, op.ev);
              const int flip = philox_uniform(P.seed, gshot, op.ev + 1) < P.pM ? 1 : 0;
              int bit = u < p0 ? 0 : 1;
              if (P.forced)  // adjoint forward pass: the outcome that reproduces the record
                bit = ((P.forced[shot * P.rec_bytes + op.idx / 8] >> (op.idx % 8)) & 1) ^ flip;
              double pb = bit == 0 ? p0 : 1.0 - p0;
              if (!P.forced && fabs(u - p0) < kNearThreshold) P.near[shot] += 1;
              P.born[shot * P.n_meas + op.idx] = pb;
              S.dmisc[D_LOGP] += log(pb);
              if (bit ^ flip) P.records[shot * P.rec_bytes + op.idx / 8] |= static_cast<uint8_t>(1u << (op.idx % 8));
              S.misc[M_OUTCOME] = bit;
              if (bit != small) set_meas_spec<T>(S, bit);
              if (P.tape_info) {
                int32_t *ti = P.tape_info + (shot * P.n_ops_total + oi) * kTapeInts;
                const int mb = S.misc[M_BIT];
                ti[0] = (mb & 3) | (S.misc[M_CASEB] << 2) | (bit << 3) | (S.misc[M_LIDX] << 4) |
                        (((mb >> 4) & 1) << 6);
              }
            }
            __syncthreads();
            caseB = S.misc[M_CASEB];
            lidx = S.misc[M_LIDX];
            outcome = S.misc[M_OUTCOME];
            tq = clock64();
            if (outcome != small) mps_prepare<T>(P, S, shot, X, a, b);
            __syncthreads();
            prof_mark(S.dmisc, PROF_LEFT, tq);
            mps_finish<T>(P, S, shot, X, a, b);
          } else {
            long long tq = clock64();
            mps_prepare<T>(P, S, shot, X, a, b);
            __syncthreads();
            prof_mark(S.dmisc, PROF_LEFT, tq);
            mps_finish<T>(P, S, shot, X, a, b);
            if (P.phi_store && P.rot_ord[oi] >= 0) {  // adjoint: keep the state after the rotation
              const int64_t slot = shot * P.n_rot + P.rot_ord[oi];
              cplx<T> *dst = reinterpret_cast<cplx<T> *>(P.phi_store) + slot * P.slab_elems;
              for (int k = 0; k < n; ++k) {
                const cplx<T> *src = site_ptr<T>(P, shot, k);
                const int64_t cnt = 2ll * S.chi[k] * S.chi[k + 1];
                for (int64_t e = tid(); e < cnt; e += kThreads) dst[P.site_off[k] + e] = src[e];
              }
              for (int e = tid(); e <= n; e += kThreads) P.phi_chi[slot * (n + 1) + e] = S.chi[e];
            }
          }
          if (meas) {
            if (caseB) tableau_caseB(S.tx, S.tz, S.tm, n, W, S.ppx, S.ppz, S.misc[M_J], lidx);
            if (tid() == 0 && op.pauli == 1) {
              if (outcome) pauli_left(S.tm, n, op.a, 1);
              if (philox_uniform(P.seed, gshot, op.ev + 2) < P.pR) pauli_left(S.tm, n, op.a, 1);
            }
          }
          break;
        }
        default:
          if (tid() == 0) S.misc[M_FAIL] = STN_EINVAL;
      }
      __syncthreads();
    }
    // store
    for (int e = tid(); e < 2 * n * W; e += kThreads) {
      P.tab_x[shot * 2 * n * W + e] = S.tx[e];
      P.tab_z[shot * 2 * n * W + e] = S.tz[e];
    }
    for (int e = tid(); e < 2 * n; e += kThreads) P.tab_m[shot * 2 * n + e] = S.tm[e];
    for (int e = tid(); e <= n; e += kThreads) P.chi[shot * (n + 1) + e] = S.chi[e];
    if (tid() == 0) {
      P.center[shot] = S.misc[M_CENTER];
      P.status[shot] = S.misc[M_FAIL];
      P.maxchi[shot] = S.misc[M_MAXCHI];
      P.disc[shot] = S.dmisc[D_DISC];
      P.logp[shot] = S.dmisc[D_LOGP];
      P.flops[shot] += S.dmisc[D_FLOPS];
      S.dmisc[D_PROF + 1 + PROF_OPS] = static_cast<double>(clock64() - t_ops);
      for (int i = 0; i < kProfSlots; ++i) P.prof[shot * kProfSlots + i] += S.dmisc[D_PROF + 1 + i];
      if (S.misc[M_FAIL]) atomicCAS(P.err, 0, S.misc[M_FAIL]);
    }
    __syncthreads();
  }
  if (tc_alloc) tc_teardown();
}

// Identity frame, |0...0>, cleared records and accumulators.
template <typename T>
__global__ void init_kernel(EngineParams P) {
  const int n = P.n, W = P.W;
  for (int64_t shot = blockIdx.x; shot < P.shots; shot += gridDim.x) {
    for (int e = tid(); e < 2 * n * W; e += blockDim.x) {
      int r = e / W, w = e % W;
      int q = r % n;
      uint64_t bit = (q >> 6) == w ? (1ull << (q & 63)) : 0ull;
      P.tab_x[shot * 2 * n * W + e] = r < n ? bit : 0ull;
      P.tab_z[shot * 2 * n * W + e] = r < n ? 0ull : bit;
    }
    for (int e = tid(); e < 2 * n; e += blockDim.x) P.tab_m[shot * 2 * n + e] = 0;
    for (int e = tid(); e <= n; e += blockDim.x) P.chi[shot * (n + 1) + e] = 1;
    cplx<T> *slab = reinterpret_cast<cplx<T> *>(P.mps) + shot * P.slab_elems;
    for (int k = tid(); k < n; k += blockDim.x) {
      slab[P.site_off[k]] = cmake<T>(1, 0);
      slab[P.site_off[k] + 1] = cmake<T>(0, 0);
    }
    for (int e = tid(); e < P.rec_bytes; e += blockDim.x) P.records[shot * P.rec_bytes + e] = 0;
    for (int e = tid(); e < P.n_meas; e += blockDim.x) P.born[shot * P.n_meas + e] = 0.0;
    if (tid() == 0) {
      P.center[shot] = 0;
      P.status[shot] = 0;
      P.maxchi[shot] = 1;
      P.near[shot] = 0;
      P.disc[shot] = 0.0;
      P.logp[shot] = 0.0;
    }
  }
}

// ---------------------------------------------------------------------------
// Kernel-level checks of the dense routines on one CTA (complex elements of
// precision T, column-major C/V for the SVD, row-major B for the QR).
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) dense_check_kernel(int what, int m, int n, cplx<T> *A,
                                                                  cplx<T> *V, T *sig2, int use_smem) {
  extern __shared__ __align__(16) char smem_raw[];
  tc_disable();
  double *red = reinterpret_cast<double *>(smem_raw);
  double *dm = red + kThreads;
  int *flag = reinterpret_cast<int *>(dm + 16);
  cplx<T> *uv = reinterpret_cast<cplx<T> *>(flag + 16);
  cplx<T> *buf = uv + kMaxVec;
  float *rv_wrk = reinterpret_cast<float *>(buf + SvdSmem<T>::elems);
  if (what == 0) {
    qr_r_inplace<T>(m, n, A, n, buf, SvdSmem<T>::elems, red, dm);
  } else if (what == 2) {
    // explicit Q of the gauge steps: reflectors kept in sig2's buffer
    cplx<T> *vstore = reinterpret_cast<cplx<T> *>(sig2);
    qr_r_inplace<T>(m, n, A, n, buf, SvdSmem<T>::elems, red, dm, vstore);
    form_q<T>(m, min(m, n), vstore, V, buf, SvdSmem<T>::elems);
  } else if (use_smem == 3) {
    // the large-bond path of the truncation sweep: A row-major (m x n),
    // R factor, Jacobi on X = R^dag (n x k), V = normalised columns of X
    qr_r_inplace<T>(m, n, A, n, buf, SvdSmem<T>::elems, red, dm);
    const int k = min(m, n);
    const bool regs = sizeof(T) == 4 && k > 16 && n <= kThreads;
    const bool x_smem = !regs && n * k <= SvdSmem<T>::elems;
    cplx<T> *Xc = x_smem ? buf : A;
    for (int e = tid(); e < n * k; e += kThreads) Xc[e] = cconj(A[e]);
    __syncthreads();
    if (x_smem) svd_onesided<T>(n, k, Xc, nullptr, sig2, flag, red);
    else svd_onesided_blocked<T>(n, k, Xc, nullptr, sig2, flag, red, buf, SvdSmem<T>::elems,
                                 regs ? rv_wrk : nullptr);
    for (int e = tid(); e < n * n; e += kThreads) {
      const int c = e / n;
      const T l = c < k ? sig2[c] : T(0);
      V[e] = l > T(0) ? cscale(Xc[e], T(1) / sqrt(l)) : cmake<T>(0, 0);
    }
    for (int c = k + tid(); c < n; c += kThreads) sig2[c] = T(0);
  } else {
    cplx<T> *C = A, *VV = V;
    if (use_smem == 1) {
      C = buf;
      VV = buf + m * n;
      for (int e = tid(); e < m * n; e += kThreads) C[e] = A[e];
      __syncthreads();
    }
    if (use_smem == 2) svd_onesided_blocked<T>(m, n, C, VV, sig2, flag, red, buf, SvdSmem<T>::elems);
    else svd_onesided<T>(m, n, C, VV, sig2, flag, red);
    if (use_smem == 1) {
      for (int e = tid(); e < m * n; e += kThreads) A[e] = C[e];
      for (int e = tid(); e < n * n; e += kThreads) V[e] = VV[e];
    }
  }
}

template <typename T>
cudaError_t launch_dense_check_t(int what, int m, int n, void *A, void *V, void *sig2, int use_smem,
                                        cudaStream_t s) {
  size_t smem = sizeof(double) * (kThreads + 16) + sizeof(int) * 16 + sizeof(cplx<T>) * kMaxVec;
  smem += sizeof(cplx<T>) * SvdSmem<T>::elems;  // QR panel, SVD matrix or staged column blocks
  smem += sizeof(float) * kRvWrkFloats;           // register-visit reductions
  cudaError_t e = cudaFuncSetAttribute(dense_check_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  dense_check_kernel<T><<<1, kThreads, smem, s>>>(what, m, n, static_cast<cplx<T> *>(A),
                                                  static_cast<cplx<T> *>(V), static_cast<T *>(sig2), use_smem);
  return cudaGetLastError();
}

// The sweeps' complex contraction alone on one CTA: C = alpha op(A) op(B) +
// beta C through cgemm, with the tensor cores set up as the round kernel
// sets them up (complex64 and use_tc) or disabled.  *status becomes
// STN_ETIMEOUT if a tensor-core wait ran out.
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) dense_gemm_kernel(int ta, int tb, int m, int n, int k, cplx<T> alpha,
                                                                 const cplx<T> *A, int lda, const cplx<T> *B, int ldb,
                                                                 cplx<T> beta, cplx<T> *C, int ldc, int use_tc,
                                                                 int *status) {
  extern __shared__ __align__(16) char smem_raw[];
  cplx<T> *tile = reinterpret_cast<cplx<T> *>(smem_raw);
  float *stage = reinterpret_cast<float *>(tile + kBK * (kBM + kPad + kBN + kPad));
  bool tc = false;
  if constexpr (sizeof(T) == 4) tc = use_tc != 0;
  if (tc) tc_setup(stage);
  else tc_disable();
  if (ta == 0 && tb == 0) cgemm<T, 0, 0>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, tile);
  else if (ta == 0) cgemm<T, 0, 1>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, tile);
  else if (tb == 0) cgemm<T, 1, 0>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, tile);
  else cgemm<T, 1, 1>(m, n, k, alpha, A, lda, B, ldb, beta, C, ldc, tile);
  if (tc) {
    if (threadIdx.x == 0 && g_tc.failed) *status = STN_ETIMEOUT;
    tc_teardown();
  }
}

template <typename T>
cudaError_t launch_dense_gemm_t(int ta, int tb, int m, int n, int k, const double *alpha, const void *A, int lda,
                                const void *B, int ldb, const double *beta, void *C, int ldc, int use_tc, int *status,
                                cudaStream_t s) {
  size_t smem = sizeof(cplx<T>) * kBK * (kBM + kPad + kBN + kPad);
  if (sizeof(T) == 4 && use_tc) smem += sizeof(float) * kTcStageFloats;
  cudaError_t e = cudaFuncSetAttribute(dense_gemm_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  cplx<T> al, be;
  al.re = static_cast<T>(alpha[0]);
  al.im = static_cast<T>(alpha[1]);
  be.re = static_cast<T>(beta[0]);
  be.im = static_cast<T>(beta[1]);
  dense_gemm_kernel<T><<<1, kThreads, smem, s>>>(ta, tb, m, n, k, al, static_cast<const cplx<T> *>(A), lda,
                                                 static_cast<const cplx<T> *>(B), ldb, be, static_cast<cplx<T> *>(C),
                                                 ldc, use_tc, status);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_init_t(const EngineParams &p, cudaStream_t s) {
  int grid = p.shots < 4096 ? p.shots : 4096;
  if (grid < 1) return cudaSuccess;
  init_kernel<T><<<grid, 128, 0, s>>>(p);
  return cudaGetLastError();
}

// ---------------------------------------------------------------------------
// Diagnostics of the current batch, one CTA per shot slot (grid-strided).
// what = DIAG_LOGICAL: out[shot] = <psi| L |psi> for L the product of
//   `letter` (1 X, 3 Z) over the nl qubits lq (Sec. II, Eq. 1: the logical
//   operator's expectation behind the P_L estimator).  L is pushed through
//   the shot's frame, P' = C^dag L C = i^m X^x Z^z (the images of the
//   commuting factors multiplied with the exact phase), the orthogonality
//   centre is moved into P''s support, and <MPS| P' |MPS> is contracted over
//   it.  A shot whose status is set gets NaN.
// what = DIAG_SCHMIDT: for shot `target` only, the centre is moved to site
//   `cut` and the squared singular values of that site as a
//   (2 chi_cut) x chi_{cut+1} matrix, the squared Schmidt coefficients across
//   the cut after site `cut` (Sec. IV B, Fig. 2), go to out[] largest first,
//   their number to *count.
// Both only move the orthogonality centre by exact gauge steps: the state,
// and every later result of the batch, are unchanged (up to rounding).
enum { DIAG_LOGICAL = 0, DIAG_SCHMIDT = 1 };

template <typename T>
__global__ void __launch_bounds__(kThreads, 1) diag_kernel(EngineParams P, int what, int target, int cut,
                                                           const int32_t *lq, int nl, int letter, double *out,
                                                           int *count) {
  extern __shared__ __align__(16) char smem_raw[];
  tc_disable();
  const int n = P.n, W = P.W;
  Smem<T> S = carve<T>(smem_raw, n, W, P.svd_elems);
  Scratch<T> X = scratch_for<T>(P, P.work_c);
  for (int64_t shot = blockIdx.x; shot < P.shots; shot += gridDim.x) {
    if (what == DIAG_SCHMIDT && shot != target) continue;
    for (int e = tid(); e < 2 * n * W; e += kThreads) {
      S.tx[e] = P.tab_x[shot * 2 * n * W + e];
      S.tz[e] = P.tab_z[shot * 2 * n * W + e];
    }
    for (int e = tid(); e < 2 * n; e += kThreads) S.tm[e] = P.tab_m[shot * 2 * n + e];
    for (int e = tid(); e <= n; e += kThreads) S.chi[e] = P.chi[shot * (n + 1) + e];
    if (tid() == 0) {
      S.misc[M_CENTER] = P.center[shot];
      S.misc[M_FAIL] = P.status[shot];
    }
    __syncthreads();
    if (S.misc[M_FAIL]) {
      if (tid() == 0) {
        if (what == DIAG_LOGICAL) out[shot] = nan("");
        else *count = 0;
      }
      __syncthreads();
      continue;
    }
    if (what == DIAG_LOGICAL) {
      if (tid() == 0) {
        for (int w = 0; w < W; ++w) S.ppx[w] = S.ppz[w] = 0;
        int m = 0;
        for (int i = 0; i < nl; ++i) {
          const int r = letter == 3 ? n + lq[i] : lq[i];
          int sw = 0;
          for (int w = 0; w < W; ++w) {
            sw += popc64(S.ppz[w] & S.tx[r * W + w]);
            S.ppx[w] ^= S.tx[r * W + w];
            S.ppz[w] ^= S.tz[r * W + w];
          }
          m += S.tm[r] + 2 * sw;
        }
        int lo = n, hi = -1;
        for (int q = 0; q < n; ++q)
          if (((S.ppx[q >> 6] | S.ppz[q >> 6]) >> (q & 63)) & 1) { lo = min(lo, q); hi = max(hi, q); }
        S.misc[M_LO] = lo;
        S.misc[M_HI] = hi;
        S.misc[M_BIT] = m & 3;
      }
      __syncthreads();
      const int lo = S.misc[M_LO], hi = S.misc[M_HI], m = S.misc[M_BIT];
      double e;
      if (lo > hi) {  // L maps to a multiple of the identity
        e = m == 0 ? 1.0 : (m == 2 ? -1.0 : 0.0);
      } else {
        const int c0 = S.misc[M_CENTER];
        const int tgt = c0 < lo ? lo : (c0 > hi ? hi : c0);
        if (tgt != c0) mps_move_center<T>(P, S, shot, X, tgt);
        e = S.misc[M_FAIL] ? nan("") : mps_expect<T>(P, S, shot, X, lo, hi, m);
      }
      if (tid() == 0) out[shot] = e;
    } else {
      mps_move_center<T>(P, S, shot, X, cut);
      const int l = S.chi[cut], r = S.chi[cut + 1], mrows = 2 * l, kx = min(mrows, r);
      int cnt = 0;
      if (!S.misc[M_FAIL] && mrows <= kMaxVec) {
        const cplx<T> *A = site_ptr<T>(P, shot, cut);
        for (int e = tid(); e < mrows * r; e += kThreads) X.y[e] = A[e];
        __syncthreads();
        qr_r_inplace<T>(mrows, r, X.y, r, S.jbuf, P.svd_elems, S.red, S.dmisc + 4);
        // Jacobi on R^dag (r x kx, column-major, ld r), in place as in the sweep
        for (int e = tid(); e < r * kx; e += kThreads) X.y[e] = cconj(X.y[e]);
        __syncthreads();
        svd_onesided_blocked<T>(r, kx, X.y, nullptr, X.lam, &S.misc[M_JFLAG], S.red, S.jbuf, P.svd_elems,
                                sizeof(T) == 4 && kx > 16 && r <= kThreads ? reinterpret_cast<float *>(S.lam)
                                                                            : nullptr);
        sort_desc<T>(kx, X.lam, S.perm);
        for (int i = tid(); i < kx; i += kThreads) out[i] = fmax(static_cast<double>(X.lam[S.perm[i]]), 0.0);
        cnt = kx;
      }
      if (tid() == 0) *count = cnt;
    }
    __syncthreads();
    for (int e = tid(); e <= n; e += kThreads) P.chi[shot * (n + 1) + e] = S.chi[e];
    if (tid() == 0) {
      P.center[shot] = S.misc[M_CENTER];
      if (S.misc[M_FAIL]) P.status[shot] = S.misc[M_FAIL];
    }
    __syncthreads();
  }
}

// ---------------------------------------------------------------------------
// <mu| phase (x)_k op_k |phi> of two MPSs over all n sites: mu is the shot's
// own MPS (bonds S.chi), phi a stored state (sites at site_off in phi, bonds
// phi_chi).  The Pauli string in S.ppx/ppz (letters X^x Z^z) acts on phi when
// with_op.  Transfer matrices E (chi_mu x chi_phi): E <- A_mu^dag (E B),
// through two GEMMs per site.  CTA-wide; returns the complex value in double.
template <typename T>
static __device__ cplx<double> mps_overlap(const EngineParams &P, const Smem<T> &S, int64_t shot, const Scratch<T> &X,
                                           const cplx<T> *phi, const int *phi_chi, bool with_op, int m) {
  const int n = P.n;
  const cplx<T> one = cmake<T>(1, 0), zero = cmake<T>(0, 0);
  MpoSpec<T> sp;
  sp.kind = MPO_ROT; sp.lo = -1; sp.hi = -1; sp.j = -1;
  sp.w0 = one; sp.w1 = one; sp.v0 = zero; sp.v1 = zero;
  for (int k = 0; k < n; ++k) {
    const cplx<T> *A = site_ptr<T>(P, shot, k);
    const int clm = S.chi[k], crm = S.chi[k + 1];
    const int clp = phi_chi[k], crp = phi_chi[k + 1];
    const cplx<T> *B = phi + P.site_off[k];
    const bool acts = with_op && (((S.ppx[k >> 6] | S.ppz[k >> 6]) >> (k & 63)) & 1);
    if (acts) {
      cplx<T> op[4];
      site_op(sp, S.ppx, S.ppz, k, 1, op);
      const int64_t tot = static_cast<int64_t>(clp) * 2 * crp;
      for (int64_t e = tid(); e < tot; e += kThreads) {
        const int r = static_cast<int>(e % crp), s2 = static_cast<int>((e / crp) % 2);
        const int64_t l = e / (2 * crp);
        cplx<T> v = zero;
        cfma(v, op[s2 * 2 + 0], B[(l * 2 + 0) * crp + r]);
        cfma(v, op[s2 * 2 + 1], B[(l * 2 + 1) * crp + r]);
        X.sa[e] = v;
      }
      __syncthreads();
      B = X.sa;
    }
    if (k == 0) {  // E = A_mu^dag B over the physical index (chi_0 = 1)
      cgemm<T, 1, 0>(crm, crp, 2 * clm, one, A, crm, B, crp, zero, X.e, crp, S.tile);
    } else {
      cgemm<T, 0, 0>(clm, 2 * crp, clp, one, X.e, clp, B, 2 * crp, zero, X.te, 2 * crp, S.tile);
      cgemm<T, 1, 0>(crm, crp, 2 * clm, one, A, crm, X.te, crp, zero, X.e, crp, S.tile);
    }
  }
  const cplx<T> v = X.e[0];
  cplx<double> r = cmake<double>(static_cast<double>(v.re), static_cast<double>(v.im));
  const cplx<double> ph = ipow<double>(m);
  r = cmul(ph, r);
  __syncthreads();
  return r;
}

// Backward pass of the adjoint (see stn_logprob_grad): one CTA per record,
// the shot's MPS holding mu (initially the final state of the forced forward
// pass), the ops walked from last to first.  At a rotation of pair k the term
// 2 Re <mu| (-i P') |phi_j> / <mu|phi_j> is added to grad[k] (phi_j the
// stored state after that rotation), then mu <- exp(+i theta P') mu; a case-A
// measurement applies its projector again, a case-B measurement applies
// U |v><0|_j; every application is followed by the truncating sweep.
// Clifford gates and Paulis only changed the frame and leave mu alone.
template <typename T>
__global__ void __launch_bounds__(kThreads, 1) adjoint_kernel(EngineParams P, double *grad) {
  extern __shared__ __align__(16) char smem_raw[];
  tc_disable();
  const int n = P.n, W = P.W;
  Smem<T> S = carve<T>(smem_raw, n, W, P.svd_elems);
  Scratch<T> X = scratch_for<T>(P, P.work_c);
  for (int64_t shot = blockIdx.x; shot < P.shots; shot += gridDim.x) {
    for (int e = tid(); e <= n; e += kThreads) S.chi[e] = P.chi[shot * (n + 1) + e];
    if (tid() == 0) {
      S.misc[M_CENTER] = P.center[shot];
      S.misc[M_FAIL] = P.status[shot];
      S.misc[M_MAXCHI] = P.maxchi[shot];
      S.dmisc[D_DISC] = 0.0;
      S.dmisc[D_FLOPS] = 0.0;
    }
    __syncthreads();
    for (int oi = P.n_ops_total - 1; oi >= 0 && !S.misc[M_FAIL]; --oi) {
      const Op op = P.ops[oi];
      if (op.kind != OP_ROT && op.kind != OP_MEAS) continue;
      const int64_t t = shot * P.n_ops_total + oi;
      const int32_t *ti = P.tape_info + t * kTapeInts;
      const int info = ti[0], lo = ti[1], hi = ti[2], jq = ti[3];
      const int m = info & 3;
      if (tid() < W) {
        S.ppx[tid()] = P.tape_px[t * W + tid()];
        S.ppz[tid()] = P.tape_pz[t * W + tid()];
      }
      __syncthreads();
      MpoSpec<T> &sp = *S.spec;
      if (op.kind == OP_ROT) {
        const int64_t slot = shot * P.n_rot + P.rot_ord[oi];
        const cplx<T> *phi = reinterpret_cast<const cplx<T> *>(P.phi_store) + slot * P.slab_elems;
        const int *phi_chi = P.phi_chi + slot * (n + 1);
        const cplx<double> num = mps_overlap<T>(P, S, shot, X, phi, phi_chi, true, m + 3);  // (-i) i^m
        const cplx<double> den = mps_overlap<T>(P, S, shot, X, phi, phi_chi, false, 0);
        if (tid() == 0) {
          const double d2 = den.re * den.re + den.im * den.im;
          const double re = (num.re * den.re + num.im * den.im) / d2;  // Re(num / den)
          if (!(d2 > 0.0) || !isfinite(re)) S.misc[M_FAIL] = STN_ENUMERIC;
          else atomicAdd(&grad[op.idx], 2.0 * re);
          const double th = P.theta[op.idx];
          sp.kind = MPO_ROT;
          sp.lo = lo; sp.hi = hi; sp.j = -1;
          sp.w0 = cmake<T>(static_cast<T>(cos(th)), 0);
          sp.w1 = cmul(cmake<T>(0, static_cast<T>(sin(th))), ipow<T>(m));  // +i sin(theta) i^m
        }
      } else if (tid() == 0) {
        const int caseB = (info >> 2) & 1, bit = (info >> 3) & 1, lidx = (info >> 4) & 3, neg = (info >> 6) & 1;
        sp.lo = lo; sp.hi = hi; sp.j = jq;
        sp.w0 = cmake<T>(1, 0);
        sp.w1 = cmake<T>(1, 0);
        if (!caseB) {  // the forward projector (I + (-1)^b P')/2 again
          const int sgn = (bit ? -1 : 1) * ((m & 2) ? -1 : 1);
          sp.kind = MPO_PROJ_Z;
          sp.par = sgn > 0 ? 0 : 1;
        } else {  // U |v><0|_j, v the lambda eigenvector of the site-j letter
          (void)neg;
          const T r2 = static_cast<T>(0.70710678118654752440);
          const bool zj = lidx >= 2;
          const bool lam_neg = lidx & 1;
          sp.kind = MPO_ADJ_B;
          sp.v0 = cmake<T>(r2, 0);
          sp.v1 = zj ? cmake<T>(0, lam_neg ? -r2 : r2) : cmake<T>(lam_neg ? -r2 : r2, 0);
        }
      }
      __syncthreads();
      if (S.misc[M_FAIL]) break;
      const int c0 = S.misc[M_CENTER];
      const int tgt = c0 < lo ? lo : (c0 > hi ? hi : c0);
      if (tgt != c0) mps_move_center<T>(P, S, shot, X, tgt);
      if (S.misc[M_FAIL]) break;
      mps_prepare<T>(P, S, shot, X, lo, hi);
      __syncthreads();
      mps_finish<T>(P, S, shot, X, lo, hi);
      __syncthreads();
    }
    for (int e = tid(); e <= n; e += kThreads) P.chi[shot * (n + 1) + e] = S.chi[e];
    if (tid() == 0) {
      P.center[shot] = S.misc[M_CENTER];
      P.status[shot] = S.misc[M_FAIL];
      if (S.misc[M_FAIL]) atomicCAS(P.err, 0, S.misc[M_FAIL]);
    }
    __syncthreads();
  }
}

template <typename T>
cudaError_t launch_adjoint_t(const EngineParams &p, double *grad, int grid, cudaStream_t s) {
  size_t smem = smem_bytes<T>(p.n, p.W, p.svd_elems);
  cudaError_t e = cudaFuncSetAttribute(adjoint_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  adjoint_kernel<T><<<grid, kThreads, smem, s>>>(p, grad);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_diag_t(const EngineParams &p, int what, int target, int cut, const int32_t *lq, int nl,
                          int letter, double *out, int *count, int grid, cudaStream_t s) {
  size_t smem = smem_bytes<T>(p.n, p.W, p.svd_elems);
  cudaError_t e = cudaFuncSetAttribute(diag_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  diag_kernel<T><<<grid, kThreads, smem, s>>>(p, what, target, cut, lq, nl, letter, out, count);
  return cudaGetLastError();
}

template <typename T>
cudaError_t launch_round_t(const EngineParams &p, int grid, cudaStream_t s) {
  size_t smem = smem_bytes<T>(p.n, p.W, p.svd_elems);
  cudaError_t e = cudaFuncSetAttribute(round_kernel<T>, cudaFuncAttributeMaxDynamicSharedMemorySize,
                                       static_cast<int>(smem));
  if (e != cudaSuccess) return e;
  round_kernel<T><<<grid, kThreads, smem, s>>>(p);
  return cudaGetLastError();
}

}  // namespace stn
