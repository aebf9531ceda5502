// Step a3 on the tensor cores (tcgen05, sm_103a): the per-degree contraction
//   c^l_{mn} = sum_s w_s f_lm(r_s) conj(h_ln(r_s))                 (Eq. sigmalmm)
// as one real matrix product per (particle, degree pair {l, L-l}):
//   D[r][j] = sum_k A[r][k] B[j][k],   k < 2S (zero-padded to a multiple of 16),
// A row of degree d, order m >= 0:  (Re f_dm(r_0..r_{S-1}), Im f_dm(r_0..r_{S-1})),
// B rows of degree d, n = -d..d:    (w Re h_dn, w Im h_dn)   -> column of Re c^d_{mn},
//                                   (-w Im h_dn, w Re h_dn)  -> column of Im c^d_{mn},
// negative orders from h_{d,-n} = (-1)^n conj(h_dn) (real volumes).  Both
// degrees of the pair share one M = 128 tile (rows 0..l, then l+1..L+1) and
// one N tile (4(L+1) columns padded to 16), so one chain of MMAs covers the
// pair; the cross blocks are computed and never read.  Operands are TF32
// (cvt.rna) or BF16 (round to nearest) in shared memory, canonical K-major
// layout without swizzle (8-row x 16-byte core matrices, K-adjacent core
// matrices 128 bytes apart); the accumulator is FP32 in tensor memory.
//
// Sequence per CTA: stage A and B (generic stores, then a proxy fence),
// allocate tensor-memory columns (one warp), one thread issues the MMAs and
// commits them to an mbarrier, all threads wait on it with an iteration
// limit (on expiry: error bit, no read of the accumulator), the warps copy
// their accumulator lanes to shared memory, the columns are freed, and the
// epilogue writes the grouped layout (see internal.cuh): c^l_{mn} from row m,
// c^l_{nm} from row n or, for n < 0, from (-1)^{m+n} conj of row -n.
#include <cuda_bf16.h>
#include <stdint.h>
#include "internal.cuh"

namespace matcha {
namespace {

constexpr int TC_THREADS = 128;  // four warps: one per 32 accumulator lanes
constexpr int TC_M = 128;
constexpr long TC_WAIT_LIMIT = 1L << 24;  // mbarrier polls before giving up

__device__ __forceinline__ uint32_t su32(const void *p) {
  return static_cast<uint32_t>(__cvta_generic_to_shared(p));
}

// Shared-memory matrix descriptor: start address, leading-dimension byte
// offset (between K-adjacent core matrices), stride-dimension byte offset
// (between M/N-adjacent core matrices), descriptor version 1, no swizzle.
__host__ __device__ __forceinline__ uint64_t smem_desc(uint32_t saddr, uint32_t lbo, uint32_t sbo) {
  uint64_t d = 0;
  d |= (uint64_t)((saddr >> 4) & 0x3FFFu);
  d |= (uint64_t)((lbo >> 4) & 0x3FFFu) << 16;
  d |= (uint64_t)((sbo >> 4) & 0x3FFFu) << 32;
  d |= (uint64_t)1 << 46;
  return d;
}

// Instruction descriptor: FP32 accumulator, A and B of format `fmt` (TF32 = 2
// under kind::tf32, BF16 = 1 under kind::f16), both K-major, N >> 3, M >> 4.
__host__ __device__ __forceinline__ uint32_t instr_desc(int fmt, int M, int N) {
  return (1u << 4) | ((uint32_t)fmt << 7) | ((uint32_t)fmt << 10) | ((uint32_t)(N >> 3) << 17) |
         ((uint32_t)(M >> 4) << 24);
}

template <int BF16> struct Op;
template <> struct Op<0> {  // TF32 in 32-bit containers
  static constexpr int bytes = 4;
  __device__ static void put(unsigned char *base, long off, float v) {
    uint32_t t;
    asm("cvt.rna.tf32.f32 %0, %1;" : "=r"(t) : "f"(v));
    *reinterpret_cast<uint32_t *>(base + off) = t;
  }
  __device__ static void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::tf32 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(id), "r"(acc));
  }
};
template <> struct Op<1> {  // BF16
  static constexpr int bytes = 2;
  __device__ static void put(unsigned char *base, long off, float v) {
    *reinterpret_cast<__nv_bfloat16 *>(base + off) = __float2bfloat16_rn(v);
  }
  __device__ static void mma(uint32_t tmem, uint64_t ad, uint64_t bd, uint32_t id, int acc) {
    asm volatile(
        "{\n\t.reg .pred p;\n\tsetp.ne.b32 p, %4, 0;\n\t"
        "tcgen05.mma.cta_group::1.kind::f16 [%0], %1, %2, %3, p;\n\t}\n" ::"r"(tmem),
        "l"(ad), "l"(bd), "r"(id), "r"(acc));
  }
};

}  // namespace

// Tile geometry shared by the launcher and the kernel.
struct TcGeom {
  int Kp, KC, SBO, RA, RAg, N, ncols;
  long a_range, b_off, b_range, d_bytes, smem;
};
__host__ __device__ inline TcGeom tc_geom(int S, int L, int bytes) {
  TcGeom g;
  g.Kp = (2 * S + 15) / 16 * 16;
  g.KC = g.Kp * bytes / 16;    // 16-byte chunks along K
  g.SBO = g.KC * 128;          // bytes between 8-row groups
  g.RA = L + 2;                // A rows used: degree l (l+1 rows) then L-l (L-l+1 rows)
  g.RAg = (g.RA + 7) / 8;
  g.N = (4 * (L + 1) + 15) / 16 * 16;
  g.ncols = 32;
  while (g.ncols < g.N) g.ncols <<= 1;
  g.a_range = (long)(TC_M / 8) * g.SBO;  // what the A descriptor spans
  g.b_off = (long)g.RAg * g.SBO;
  g.b_range = (long)(g.N / 8) * g.SBO;
  g.d_bytes = 4L * g.RA * g.N;
  long s = g.b_off + g.b_range;
  if (g.a_range > s) s = g.a_range;
  if (g.d_bytes > s) s = g.d_bytes;
  g.smem = (s + 1023) / 1024 * 1024;
  return g;
}
bool correlate_tc_fits(int S, int L, int bytes) {
  TcGeom g = tc_geom(S, L, bytes);
  return g.N <= 256 && g.RA <= TC_M && g.smem <= 200 * 1024;
}

namespace {

template <int BF16>
__global__ void __launch_bounds__(TC_THREADS)
    k_correlate_tc(const float *__restrict__ f, const float *__restrict__ h, int S, int L,
                   long h_stride, const double *__restrict__ wrad, long nc, float *__restrict__ c,
                   int *__restrict__ err) {
  using O = Op<BF16>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  const TcGeom G = tc_geom(S, L, O::bytes);
  const long b = blockIdx.y;
  const int nlm = (L + 1) * (L + 2) / 2;
  const float *fb = f + 2 * b * (long)S * nlm;
  const float *hb = h + 2 * (b * h_stride) * (long)S * nlm;
  float *cb = c + 4 * b * nc;
  const int d0 = blockIdx.x, d1 = L - blockIdx.x;
  const int nd = d0 == d1 ? 1 : 2;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  unsigned char *As = smem_raw, *Bs = smem_raw + G.b_off;
  constexpr int E = 16 / O::bytes;  // elements per 16-byte chunk
  auto off = [&](int r, int k) -> long {
    return (long)(r >> 3) * G.SBO + (long)(k / E) * 128 + (r & 7) * 16 + (k % E) * O::bytes;
  };
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  // zero the K padding of the used rows and the padded B rows
  for (int t = tid; t < G.RA * (G.Kp - 2 * S); t += TC_THREADS) {
    int r = t / (G.Kp - 2 * S), k = 2 * S + t % (G.Kp - 2 * S);
    O::put(As, off(r, k), 0.0f);
  }
  for (int t = tid; t < G.N * (G.Kp - 2 * S); t += TC_THREADS) {
    int r = t / (G.Kp - 2 * S), k = 2 * S + t % (G.Kp - 2 * S);
    O::put(Bs, off(r, k), 0.0f);
  }
  for (int t = tid; t < (G.N - 4 * (L + 1)) * 2 * S; t += TC_THREADS) {
    int r = 4 * (L + 1) + t / (2 * S), k = t % (2 * S);
    O::put(Bs, off(r, k), 0.0f);
  }
  // stage A and B: item (degree, shell s, order) reads one complex coefficient
  int r0 = 0, cbase = 0;
  for (int dd = 0; dd < 2; ++dd) {
    const int d = dd ? d1 : d0;
    const int lm0 = d * (d + 1) / 2, no = d + 1;
    if (dd == 0 || nd == 2) {
      for (int t = tid; t < S * no; t += TC_THREADS) {
        const int s = t / no, m = t - s * no;
        const float *q = fb + 2 * ((long)s * nlm + lm0 + m);
        O::put(As, off(r0 + m, s), q[0]);
        O::put(As, off(r0 + m, S + s), q[1]);
      }
      const int w2 = 2 * d + 1;
      for (int t = tid; t < S * w2; t += TC_THREADS) {
        const int s = t / w2, ni = t - s * w2, n = ni - d, an = n < 0 ? -n : n;
        const float *q = hb + 2 * ((long)s * nlm + lm0 + an);
        const float w = (float)wrad[s];
        float hr = q[0], hi = q[1];
        if (n < 0) {  // (-1)^n conj(h)
          if (an & 1) hr = -hr; else hi = -hi;
        }
        O::put(Bs, off(cbase + ni, s), w * hr);
        O::put(Bs, off(cbase + ni, S + s), w * hi);
        O::put(Bs, off(cbase + w2 + ni, s), -w * hi);
        O::put(Bs, off(cbase + w2 + ni, S + s), w * hr);
      }
    } else {  // single-degree CTA: the second block of B stays defined (zeros)
      const int w2 = 2 * d + 1;
      for (int t = tid; t < 2 * w2 * 2 * S; t += TC_THREADS)
        O::put(Bs, off(cbase + t / (2 * S), t % (2 * S)), 0.0f);
    }
    r0 = d0 + 1;
    cbase = 2 * (2 * d0 + 1);
  }
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  __syncthreads();
  // tensor-memory columns for the accumulator
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_base)),
                 "r"(G.ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (tid == 0) {
    const uint32_t id = instr_desc(BF16 ? 1 : 2, TC_M, G.N);
    const uint32_t a0 = su32(As), b0 = su32(Bs);
    const int kstep_bytes = 32;  // K per MMA: 8 TF32 or 16 BF16 = two 16-byte chunks
    const int nk = G.Kp * O::bytes / kstep_bytes;
    for (int ks = 0; ks < nk; ++ks)
      O::mma(tmem, smem_desc(a0 + ks * 256, 128, G.SBO), smem_desc(b0 + ks * 256, 128, G.SBO), id,
             ks > 0);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     su32(&mbar))
                 : "memory");
  }
  // wait for the MMAs (bounded)
  uint32_t done = 0;
  for (long it = 0; it < TC_WAIT_LIMIT && !done; ++it)
    asm volatile(
        "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
        "selp.u32 %0, 1, 0, p;\n\t}\n"
        : "=r"(done)
        : "r"(su32(&mbar)), "r"(0)
        : "memory");
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const int ok = __syncthreads_and(done);
  float *Dt = reinterpret_cast<float *>(smem_raw);  // [RA][N], over the operands
  if (ok && 32 * warp < G.RA) {
    const int row = 32 * warp + lane;
    for (int cc = 0; cc < G.N; cc += 16) {
      uint32_t v[16];
      asm volatile(
          "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
          : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
            "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
            "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
          : "r"(tmem + ((uint32_t)(32 * warp) << 16) + (uint32_t)cc));
      asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
      if (row < G.RA)
#pragma unroll
        for (int i = 0; i < 16; ++i) Dt[(long)row * G.N + cc + i] = __uint_as_float(v[i]);
    }
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G.ncols));
  if (!ok) {
    if (tid == 0) atomicOr(err, 1);
    return;
  }
  // epilogue: one thread per partner group (m, j) of each degree
  r0 = 0;
  cbase = 0;
  for (int dd = 0; dd < nd; ++dd) {
    const int d = dd ? d1 : d0;
    const int cre = cbase, cim = cbase + 2 * d + 1;
    const float *Dr = Dt + (long)r0 * G.N;
    const int ng = (d + 1) * (d + 2) / 2;
    for (int g = tid; g < ng; g += TC_THREADS) {
      const int m = tri_floor(g), j = g - m * (m + 1) / 2;
      float e[8];
      for (int hh = 0; hh < 2; ++hh) {
        const int n = 2 * j - m + hh;
        float a = 0, bq = 0, cr = 0, ci = 0;
        if (n <= m) {
          a = Dr[(long)m * G.N + cre + n + d];
          bq = Dr[(long)m * G.N + cim + n + d];
          if (n >= 0) {
            cr = Dr[(long)n * G.N + cre + m + d];
            ci = Dr[(long)n * G.N + cim + m + d];
          } else {  // c_{n m} = (-1)^{m+n} conj(c_{-n,-m})
            const float sg = ((m + n) & 1) ? -1.0f : 1.0f;
            cr = sg * Dr[(long)(-n) * G.N + cre - m + d];
            ci = -sg * Dr[(long)(-n) * G.N + cim - m + d];
          }
        }
        e[hh] = a; e[2 + hh] = bq; e[4 + hh] = cr; e[6 + hh] = ci;
      }
      // entry (group, d): goff(m, j) + d - m, 8 reals
      const long t = (long)m * (m + 1) / 2;
      const long go = (long)(L + 2) * t - (long)m * (m + 1) * (2 * m + 1) / 6 + (long)j * (L - m + 1);
      float4 *o = reinterpret_cast<float4 *>(cb + 8 * (go + d - m));
      o[0] = make_float4(e[0], e[1], e[2], e[3]);
      o[1] = make_float4(e[4], e[5], e[6], e[7]);
    }
    r0 = d0 + 1;
    cbase = 2 * (2 * d0 + 1);
  }
}

}  // namespace

cudaError_t launch_correlate_tc(const Plan &p, const float *f, const float *h, int B, int hstride,
                                float *c, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  const int bf16 = p.tc == 2;
  const TcGeom g = tc_geom(p.S, p.LJ, bf16 ? 2 : 4);
  if (!correlate_tc_fits(p.S, p.LJ, bf16 ? 2 : 4)) return cudaErrorInvalidConfiguration;
  const dim3 grid(p.LJ / 2 + 1, B);
  if (bf16) {
    cudaFuncSetAttribute(k_correlate_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    k_correlate_tc<1><<<grid, TC_THREADS, g.smem, st>>>(f, h, p.S, p.LJ, hstride, p.wrad, p.nc, c,
                                                        p.dev_err);
  } else {
    cudaFuncSetAttribute(k_correlate_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)g.smem);
    k_correlate_tc<0><<<grid, TC_THREADS, g.smem, st>>>(f, h, p.S, p.LJ, hstride, p.wrad, p.nc, c,
                                                        p.dev_err);
  }
  return cudaGetLastError();
}

}  // namespace matcha
