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
// Persistent CTAs (two per SM, each holding 256 tensor-memory columns for its
// lifetime) walk the items (particle, degree pair) with two operand buffers:
// the operands of the next item are staged (generic stores, proxy fence)
// while the MMAs of the current one run; one thread issues the MMAs and
// commits them to an mbarrier; all threads wait on it with an iteration
// limit (on expiry: error bit, the CTA stops); warps 0-3 copy their
// accumulator lanes into the buffer the finished MMAs read; the next item's
// MMAs are issued; and the epilogue writes the grouped layout (see
// internal.cuh) while they run: c^l_{mn} from row m, c^l_{nm} from row n or,
// for n < 0, from (-1)^{m+n} conj of row -n.
#include <cuda_bf16.h>
#include <stdint.h>
#include "internal.cuh"

namespace matcha {
namespace {

constexpr int TC_THREADS = 256;  // warps 0-3 own the 128 accumulator lanes
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

// Tile geometry shared by the launcher and the kernel.  One operand buffer
// holds A's used row groups followed by B; the A descriptor spans 128 rows,
// which reach into B (rows past L+1 are never read back).  The accumulator
// tile copied out of tensor memory reuses the buffer whose MMAs are done.
struct TcGeom {
  int Kp, KC, SBO, RA, RAg, N, DS, ncols;
  long a_range, b_off, b_range, d_bytes, buf;
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
  g.DS = g.N + 1;  // odd row stride of the accumulator copy (no bank conflicts)
  g.d_bytes = 4L * g.RA * g.DS;
  long s = g.b_off + g.b_range;
  if (g.a_range > s) s = g.a_range;
  if (g.d_bytes > s) s = g.d_bytes;
  g.buf = (s + 1023) / 1024 * 1024;
  return g;
}
// Two operand buffers; at least 77 KB so that no more than two CTAs share an
// SM (each holds 256 of the SM's 512 tensor-memory columns for its lifetime).
__host__ __device__ inline long tc_smem(const TcGeom &g) {
  long s = 2 * g.buf;
  return s < 77 * 1024 ? 77 * 1024 : s;
}
bool correlate_tc_fits(int S, int L, int bytes) {
  TcGeom g = tc_geom(S, L, bytes);
  return g.N <= 256 && g.RA <= TC_M && g.ncols <= 256 && tc_smem(g) <= 200 * 1024;
}

namespace {

// Persistent CTAs, each over items (particle, degree pair) blockIdx.x,
// blockIdx.x + gridDim.x, ...; software pipeline per item i:
//   stage operands of i+1 (other buffer)   | MMAs of i run
//   wait for i, copy the accumulator to shared memory
//   issue the MMAs of i+1                   | epilogue of i (global stores)
template <int BF16>
__global__ void __launch_bounds__(TC_THREADS, 1)
    k_correlate_tc(const float *__restrict__ f, const float *__restrict__ h, int S, int L,
                   long h_stride, const double *__restrict__ wrad, long nc, float *__restrict__ c,
                   int B, int *__restrict__ err, long wait_limit) {
  using O = Op<BF16>;
  extern __shared__ __align__(1024) unsigned char smem_raw[];
  __shared__ __align__(8) uint64_t mbar;
  __shared__ uint32_t tmem_base;
  __shared__ float wsh[128];
  const TcGeom G = tc_geom(S, L, O::bytes);
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nlm = (L + 1) * (L + 2) / 2;
  const int npair = L / 2 + 1;
  const long nitems = (long)B * npair;
  const long first = blockIdx.x;
  const int nmine = first < nitems ? (int)((nitems - 1 - first) / gridDim.x + 1) : 0;
  constexpr int E = 16 / O::bytes;  // elements per 16-byte chunk
  auto off = [&](int r, int k) -> long {
    return (long)(r >> 3) * G.SBO + (long)(k / E) * 128 + (r & 7) * 16 + (k % E) * O::bytes;
  };
  auto bufp = [&](int i) { return smem_raw + (i & 1) * G.buf; };
  for (int s = tid; s < S; s += TC_THREADS) wsh[s] = (float)wrad[s];
  if (tid == 0) {
    asm volatile("mbarrier.init.shared::cta.b64 [%0], 1;" ::"r"(su32(&mbar)));
    asm volatile("fence.mbarrier_init.release.cluster;");
  }
  const int kpad = G.Kp - 2 * S;
  __syncthreads();

  // Operands of item `it` into buffer `u`.  The K padding of every row is
  // zeroed each time (the accumulator copy of an earlier item may have
  // overwritten it); rows and columns that are never read back (A rows past
  // L+1, B rows past 4(L+1), the second block of the single-degree item
  // l = L/2) may hold anything: they reach only unread accumulator entries.
  auto stage = [&](long it, int u) {
    const long b = it / npair;
    const int q = (int)(it - b * npair);
    const int d0 = q, d1 = L - q, nd = d0 == d1 ? 1 : 2;
    const float *fb = f + 2 * b * (long)S * nlm;
    const float *hb = h + 2 * (b * h_stride) * (long)S * nlm;
    unsigned char *As = bufp(u), *Bs = As + G.b_off;
    for (int t = tid; t < G.RA * kpad; t += TC_THREADS)
      O::put(As, off(t / kpad, 2 * S + t % kpad), 0.0f);
    for (int t = tid; t < G.N * kpad; t += TC_THREADS)
      O::put(Bs, off(t / kpad, 2 * S + t % kpad), 0.0f);
    int r0 = 0, cbase = 0;
    for (int dd = 0; dd < nd; ++dd) {
      const int d = dd ? d1 : d0;
      const int lm0 = d * (d + 1) / 2, no = d + 1, w2 = 2 * d + 1;
      // item (s, m): f_dm(r_s) -> A row m; h_dm(r_s) -> the B rows of n = m and
      // n = -m.  Items go in tiles of 8 orders x 4 shells, a warp per tile, so
      // a warp's stores fall in 32 distinct banks; all loads of a round are
      // issued before any store.
      const int mt = (no + 7) >> 3;
      const int na = mt * ((S + 3) >> 2) * 32;
      const FastDiv dv(mt);
      auto item = [&](int t, int &s, int &m) {
        const int T = t >> 5, ln = t & 31, ts = dv.div(T);
        m = ((T - ts * mt) << 3) + (ln & 7);
        s = (ts << 2) + (ln >> 3);
        return m < no && s < S;
      };
      for (int t0 = tid; t0 < na; t0 += 8 * TC_THREADS) {
        float2 fv[8], hv[8];
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int t = t0 + k * TC_THREADS;
          int s, m;
          if (t < na && item(t, s, m)) {
            const long o = 2 * ((long)s * nlm + lm0 + m);
            fv[k] = __ldg(reinterpret_cast<const float2 *>(fb + o));
            hv[k] = __ldg(reinterpret_cast<const float2 *>(hb + o));
          }
        }
#pragma unroll
        for (int k = 0; k < 8; ++k) {
          const int t = t0 + k * TC_THREADS;
          int s, m;
          if (t < na && item(t, s, m)) {
            O::put(As, off(r0 + m, s), fv[k].x);
            O::put(As, off(r0 + m, S + s), fv[k].y);
            const float w = wsh[s], hr = w * hv[k].x, hi = w * hv[k].y;
            const int rp = cbase + d + m;  // n = m
            O::put(Bs, off(rp, s), hr);
            O::put(Bs, off(rp, S + s), hi);
            O::put(Bs, off(rp + w2, s), -hi);
            O::put(Bs, off(rp + w2, S + s), hr);
            if (m > 0) {  // n = -m: (-1)^m conj(h)
              const float sr = (m & 1) ? -hr : hr, si = (m & 1) ? hi : -hi;
              const int rn = cbase + d - m;
              O::put(Bs, off(rn, s), sr);
              O::put(Bs, off(rn, S + s), si);
              O::put(Bs, off(rn + w2, s), -si);
              O::put(Bs, off(rn + w2, S + s), sr);
            }
          }
        }
      }
      r0 = d0 + 1;
      cbase = 2 * (2 * d0 + 1);
    }
  };
  const uint32_t id = instr_desc(BF16 ? 1 : 2, TC_M, G.N);
  const int nk = G.Kp * O::bytes / 32;  // K per MMA: 8 TF32 or 16 BF16 = two 16-byte chunks
  auto issue = [&](int u) {             // one thread
    const uint32_t a0 = su32(bufp(u)), b0 = a0 + (uint32_t)G.b_off;
    for (int ks = 0; ks < nk; ++ks)
      O::mma(tmem_base, smem_desc(a0 + ks * 256, 128, G.SBO), smem_desc(b0 + ks * 256, 128, G.SBO),
             id, ks > 0);
    asm volatile("tcgen05.commit.cta_group::1.mbarrier::arrive::one.shared::cluster.b64 [%0];" ::"r"(
                     su32(&mbar))
                 : "memory");
  };

  // tensor-memory columns for the accumulator, held for the CTA's lifetime
  if (warp == 0) {
    asm volatile("tcgen05.alloc.cta_group::1.sync.aligned.shared::cta.b32 [%0], %1;" ::"r"(
                     su32(&tmem_base)),
                 "r"(G.ncols));
    asm volatile("tcgen05.relinquish_alloc_permit.cta_group::1.sync.aligned;");
  }
  if (nmine > 0) stage(first, 0);
  asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
  const uint32_t tmem = tmem_base;
  if (tid == 0 && nmine > 0) issue(0);

  int ok = 1, fail_i = -1;
  for (int i = 0; i < nmine && ok; ++i) {
    const long it = first + (long)i * gridDim.x;
    if (i + 1 < nmine) stage(it + gridDim.x, (i + 1) & 1);
    uint32_t done = 0;
    for (long w = 0; w < wait_limit && !done; ++w)
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}\n"
          : "=r"(done)
          : "r"(su32(&mbar)), "r"((uint32_t)(i & 1))
          : "memory");
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    float *Dt = reinterpret_cast<float *>(bufp(i));  // MMAs of item i are done with it
    if (__syncthreads_and(done) == 0) {
      ok = 0;
      fail_i = i;
      break;
    }
    if (32 * (warp & 3) < G.RA) {
      // warps w and w + 4 read lanes 32 (w % 4) .. + 31 (rows), alternate
      // 16-column chunks of them
      const int row = 32 * (warp & 3) + lane;
      const uint32_t ta = tmem + ((uint32_t)(32 * (warp & 3)) << 16);
      for (int cc = 16 * (warp >> 2); cc < G.N; cc += 32) {
        uint32_t v[16];
        asm volatile(
            "tcgen05.ld.sync.aligned.32x32b.x16.b32 {%0,%1,%2,%3,%4,%5,%6,%7,%8,%9,%10,%11,%12,%13,%14,%15}, [%16];\n"
            : "=r"(v[0]), "=r"(v[1]), "=r"(v[2]), "=r"(v[3]), "=r"(v[4]), "=r"(v[5]), "=r"(v[6]),
              "=r"(v[7]), "=r"(v[8]), "=r"(v[9]), "=r"(v[10]), "=r"(v[11]), "=r"(v[12]),
              "=r"(v[13]), "=r"(v[14]), "=r"(v[15])
            : "r"(ta + (uint32_t)cc));
        asm volatile("tcgen05.wait::ld.sync.aligned;" ::: "memory");
        if (row < G.RA)
#pragma unroll
          for (int k = 0; k < 16; ++k) Dt[(long)row * G.DS + cc + k] = __uint_as_float(v[k]);
      }
    }
    asm volatile("fence.proxy.async.shared::cta;" ::: "memory");
    asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
    __syncthreads();
    asm volatile("tcgen05.fence::after_thread_sync;" ::: "memory");
    if (tid == 0 && i + 1 < nmine) issue((i + 1) & 1);
    // epilogue of item i: one thread per partner group (m, j) of each degree
    {
      const long b = it / npair;
      const int q = (int)(it - b * npair);
      const int d0 = q, d1 = L - q, nd = d0 == d1 ? 1 : 2;
      float *cb = c + 4 * b * nc;
      int r0 = 0, cbase = 0;
      for (int dd = 0; dd < nd; ++dd) {
        const int d = dd ? d1 : d0;
        const int cre = cbase, cim = cbase + 2 * d + 1;
        const float *Dr = Dt + (long)r0 * G.DS;
        const int ng = (d + 1) * (d + 2) / 2;
        for (int g = tid; g < ng; g += TC_THREADS) {
          const int m = tri_floor(g), j = g - m * (m + 1) / 2;
          float e[8];
#pragma unroll
          for (int hh = 0; hh < 2; ++hh) {
            const int n = 2 * j - m + hh;
            float a = 0, bq = 0, cr = 0, ci = 0;
            if (n <= m) {
              a = Dr[(long)m * G.DS + cre + n + d];
              bq = Dr[(long)m * G.DS + cim + n + d];
              if (n >= 0) {
                cr = Dr[(long)n * G.DS + cre + m + d];
                ci = Dr[(long)n * G.DS + cim + m + d];
              } else {  // c_{n m} = (-1)^{m+n} conj(c_{-n,-m})
                const float sg = ((m + n) & 1) ? -1.0f : 1.0f;
                cr = sg * Dr[(long)(-n) * G.DS + cre - m + d];
                ci = -sg * Dr[(long)(-n) * G.DS + cim - m + d];
              }
            }
            e[hh] = a; e[2 + hh] = bq; e[4 + hh] = cr; e[6 + hh] = ci;
          }
          // entry (group, d): goff(m, j) + d - m, 8 reals
          const long t = (long)m * (m + 1) / 2;
          const long go =
              (long)(L + 2) * t - (long)m * (m + 1) * (2 * m + 1) / 6 + (long)j * (L - m + 1);
          float4 *o = reinterpret_cast<float4 *>(cb + 8 * (go + d - m));
          o[0] = make_float4(e[0], e[1], e[2], e[3]);
          o[1] = make_float4(e[4], e[5], e[6], e[7]);
        }
        r0 = d0 + 1;
        cbase = 2 * (2 * d0 + 1);
      }
    }
    __syncthreads();  // the accumulator copy and the buffer are free for item i + 2
  }
  if (!ok) {
    if (tid == 0) atomicOr(err, 1);
    // the MMAs of item fail_i are still in flight: wait for them (bounded)
    // before the columns they write are freed
    uint32_t done = 0;
    for (long w = 0; w < TC_WAIT_LIMIT && !done; ++w)
      asm volatile(
          "{\n\t.reg .pred p;\n\tmbarrier.try_wait.parity.shared::cta.b64 p, [%1], %2;\n\t"
          "selp.u32 %0, 1, 0, p;\n\t}\n"
          : "=r"(done)
          : "r"(su32(&mbar)), "r"((uint32_t)(fail_i & 1))
          : "memory");
  }
  asm volatile("tcgen05.fence::before_thread_sync;" ::: "memory");
  __syncthreads();
  if (warp == 0)
    asm volatile("tcgen05.dealloc.cta_group::1.sync.aligned.b32 %0, %1;" ::"r"(tmem), "r"(G.ncols));
}

}  // namespace

cudaError_t launch_correlate_tc(const Plan &p, const float *f, const float *h, int B, int hstride,
                                float *c, cudaStream_t st) {
  if (B == 0) return cudaSuccess;
  const int bf16 = p.tc == 2;
  const TcGeom g = tc_geom(p.S, p.LJ, bf16 ? 2 : 4);
  if (!correlate_tc_fits(p.S, p.LJ, bf16 ? 2 : 4) || p.S > 128) return cudaErrorInvalidConfiguration;
  static int nsm = 0;
  if (!nsm) {
    int dev = 0;
    cudaGetDevice(&dev);
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
    if (nsm <= 0) nsm = 1;
  }
  const long items = (long)B * (p.LJ / 2 + 1);
  const long per_sm = p.tune_tc_ctas == 1 ? 1 : 2;
  const int grid = (int)(items < per_sm * nsm ? items : per_sm * nsm);
  const size_t smem = (size_t)tc_smem(g);
  const long wait_limit = p.wait_limit >= 0 ? p.wait_limit : TC_WAIT_LIMIT;
  if (bf16) {
    cudaFuncSetAttribute(k_correlate_tc<1>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_correlate_tc<1><<<grid, TC_THREADS, smem, st>>>(f, h, p.S, p.LJ, hstride, p.wrad, p.nc, c, B,
                                                      p.dev_err, wait_limit);
  } else {
    cudaFuncSetAttribute(k_correlate_tc<0>, cudaFuncAttributeMaxDynamicSharedMemorySize, (int)smem);
    k_correlate_tc<0><<<grid, TC_THREADS, smem, st>>>(f, h, p.S, p.LJ, hstride, p.wrad, p.nc, c, B,
                                                      p.dev_err, wait_limit);
  }
  return cudaGetLastError();
}

}  // namespace matcha
