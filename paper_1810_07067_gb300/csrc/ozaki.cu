// FP64-accurate products on BF16 tensor cores.
//
// Every row of A (and every column of Y) is scaled by a power of two sigma so
// that |a/sigma| < 1/2, then written exactly as a/sigma = sum_{s=1..8} d_s 2^{-7s}
// with integer digits |d_s| <= 64 (8 signed 7-bit digits, 56 bits; bf16 holds
// them exactly).  Then
//   sum_k a_ik y_kj = sigma_i tau_j sum_{s,t} 2^{-7(s+t)} sum_k d_s(ik) e_t(kj),
// where the digit products are exact in FP32 and, for a fixed level s + t,
// their sums over 256 values of k stay below 2^24 and hence exact as well.
// Levels s + t <= 9 are kept (36 digit products per real product; the dropped
// part is below 2^-68 of |a||y| per term).  Tensor memory holds one FP32
// accumulator per level and per real/imaginary part (8 x 2 x jt columns, jt
// the job tile of 16 or 32 right-hand-side columns); every 256 values of k
// they are drained into FP64 registers.
// Operand tiles are stored in global memory in the shared-memory layout of the
// MMA (no-swizzle K-major core matrices), so each 16-wide k-tile is a single
// bulk asynchronous copy (TMA), double-buffered behind mbarriers.
#include <cstdio>
#include "ozaki.cuh"
#include "tc.cuh"

#define OZ_ATILE (OZ_RT * OZ_KT)          // bf16 elements per slice tile of A
#define OZ_ABLOCK (2 * OZ_S * OZ_ATILE)   // per (row tile, k-tile): re/im x 8 slices
// slice tile and block of Y for a job tile of jt right-hand-side columns
__host__ __device__ constexpr int oz_ytile(int jt) { return jt * OZ_KT; }
__host__ __device__ constexpr int oz_yblock(int jt) { return 2 * OZ_S * jt * OZ_KT; }

size_t ozaki_matrix_slices_elems(int npad, int batch) {
  return (size_t)batch * (npad / OZ_RT) * (npad / OZ_KT) * OZ_ABLOCK;
}
size_t ozaki_vector_slices_elems(int npad, int batch, int njt, int jt) {
  return (size_t)batch * njt * (npad / OZ_KT) * oz_yblock(jt);
}

// offset of element (row r, k) inside a slice tile with R rows and 16 columns
// (core matrices of 8 x 8, row-group major; two core matrices along k)
__device__ __forceinline__ int core_off(int r, int k) { return ((r >> 3) * 2 + (k >> 3)) * 64 + (r & 7) * 8 + (k & 7); }

__device__ __forceinline__ void digits(double v, float* d) {
  // v in (-1/2, 1/2): the fixed-point integer F = round(v 2^56) (|F| < 2^55),
  // written in balanced base 128 from the least significant digit up:
  // d = ((F + 64) mod 128) - 64, F <- (F - d) / 128; the leading digit ends in
  // [-64, 64].  v = sum_s d_s 2^{-7s} + (rounding < 2^{-57}).
  long long F = __double2ll_rn(v * 72057594037927936.0);  // 2^56
#pragma unroll
  for (int s = OZ_S - 1; s >= 1; --s) {
    long long dd = ((F + 64) & 127) - 64;
    d[s] = (float)dd;
    F = (F - dd) >> 7;
  }
  d[0] = (float)F;
}

__device__ __forceinline__ double pow2_scale(double mx) {
  if (!(mx > 0.0)) return 1.0;
  int e;
  frexp(mx, &e);               // mx = f 2^e, f in [1/2, 1)
  return ldexp(1.0, e + 1);    // |a| / scale < 1/2
}

// thread per (row i, group of 8 consecutive k): 16 digit rows of 16 bytes.
// The 16 values are held as fixed-point integers F = round(v 2^56) and
// written in balanced base 128 from the least significant digit up, as in
// digits(), on two 28-bit halves in 32-bit integer arithmetic:
// d = ((F + 64) mod 128) - 64, F <- (F - d) / 128; the low half's carry joins
// the high half, and the top digit ends in [-64, 64].  v = sum_s d_s 2^{-7(s+1)}
// up to the rounding of F.
__device__ __forceinline__ void digits28(long long F, int* d) {
  int lo = (int)(F & 0xFFFFFFFll), hi = (int)(F >> 28);
#pragma unroll
  for (int s = OZ_S - 1; s >= OZ_S / 2; --s) {
    const int dd = ((lo + 64) & 127) - 64;
    d[s] = dd;
    lo = (lo - dd) >> 7;
  }
  hi += lo;  // carry of the low half (0 or 1)
#pragma unroll
  for (int s = OZ_S / 2 - 1; s >= 1; --s) {
    const int dd = ((hi + 64) & 127) - 64;
    d[s] = dd;
    hi = (hi - dd) >> 7;
  }
  d[0] = hi;
}

__global__ void __launch_bounds__(128) oz_slice_matrix_kernel(const cd* __restrict__ A, int n, int npad,
                                                              const double* __restrict__ rowscale,
                                                              __nv_bfloat16* __restrict__ Asl) {
  const int b = blockIdx.z;
  const int i = blockIdx.x * blockDim.x + threadIdx.x;   // row
  const int kg = blockIdx.y;                              // group of 8 columns
  if (i >= npad) return;
  const int nrt = npad / OZ_RT, nkt = npad / OZ_KT;
  const double inv = 72057594037927936.0 / rowscale[(size_t)b * npad + i];  // 2^56 / scale
  int dr[8][OZ_S], di[8][OZ_S];
  const cd* M = A + (size_t)b * n * n;
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    int k = kg * 8 + c;
    cd v = (i < n && k < n) ? M[(size_t)k * n + i] : C(0.0);
    digits28(__double2ll_rn(v.x * inv), dr[c]);
    digits28(__double2ll_rn(v.y * inv), di[c]);
  }
  const int rt = i / OZ_RT, r = i % OZ_RT, kt = (kg * 8) / OZ_KT, kk = (kg * 8) % OZ_KT;
  __nv_bfloat16* blk = Asl + (((size_t)b * nrt + rt) * nkt + kt) * OZ_ABLOCK;
  const int off = core_off(r, kk);
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    __align__(16) __nv_bfloat16 re[8], im[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      re[c] = __float2bfloat16((float)dr[c][s]);
      im[c] = __float2bfloat16((float)di[c][s]);
    }
    *(uint4*)(blk + (0 * OZ_S + s) * OZ_ATILE + off) = *(uint4*)re;
    *(uint4*)(blk + (1 * OZ_S + s) * OZ_ATILE + off) = *(uint4*)im;
  }
}

void ozaki_slice_matrix(const cd* A, int n, int npad, int batch, __nv_bfloat16* Asl, const double* rowscale,
                        cudaStream_t s) {
  oz_slice_matrix_kernel<<<dim3((npad + 127) / 128, npad / 8, batch), 128, 0, s>>>(A, n, npad, rowscale, Asl);
}

// Y for mode m, job g: column j of [y_{+m} (nrhs jobs), D_c y_{-m} (nrhs jobs)]
__device__ __forceinline__ bool job_vec(int m, int M, int nrhs, int g, int* q, int* ridx, bool* neg) {
  if (g >= 2 * nrhs || (m == 0 && g >= nrhs)) return false;
  *neg = g >= nrhs;
  *ridx = *neg ? g - nrhs : g;
  *q = *neg ? M - m : M + m;
  return true;
}

// column scales: one block per (mode, job)
__global__ void oz_colscale_kernel(const cd* __restrict__ y, int n, int M, int nrhs, int njt, int jt,
                                   double* __restrict__ colscale) {
  const int m = blockIdx.y, g = blockIdx.x;
  int q = 0, ridx = 0;
  bool neg = false;
  const bool valid = job_vec(m, M, nrhs, g, &q, &ridx, &neg);
  const cd* v = valid ? y + ((size_t)q * nrhs + ridx) * n : nullptr;
  __shared__ double red[32];
  double mx = 0.0;
  if (valid)
    for (int k = threadIdx.x; k < n; k += blockDim.x) mx = fmax(mx, fmax(fabs(v[k].x), fabs(v[k].y)));
  for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
  if ((threadIdx.x & 31) == 0) red[threadIdx.x >> 5] = mx;
  __syncthreads();
  if (threadIdx.x < 32) {
    mx = (threadIdx.x < (blockDim.x >> 5)) ? red[threadIdx.x] : 0.0;
    for (int o = 16; o > 0; o >>= 1) mx = fmax(mx, __shfl_xor_sync(0xffffffffu, mx, o));
    if (threadIdx.x == 0) colscale[(size_t)m * njt * jt + g] = pow2_scale(mx);
  }
}

// digits: thread per (mode, job, group of 8 consecutive k); 16-byte stores
__global__ void oz_slice_vectors_kernel(const cd* __restrict__ y, int n, int npad, int M, int nrhs, int njt, int jtw,
                                        const double* __restrict__ colscale, __nv_bfloat16* __restrict__ Ysl) {
  const int m = blockIdx.y;
  const int t = blockIdx.x * blockDim.x + threadIdx.x;
  const int ngroups = npad / 8;
  const int g = t / ngroups, kg = t % ngroups;  // consecutive threads: consecutive k groups of one job
  if (g >= njt * jtw) return;
  int q = 0, ridx = 0;
  bool neg = false;
  const bool valid = job_vec(m, M, nrhs, g, &q, &ridx, &neg);
  const double inv = 1.0 / colscale[(size_t)m * njt * jtw + g];
  float dre[8][OZ_S], dim_[8][OZ_S];
#pragma unroll
  for (int c = 0; c < 8; ++c) {
    const int k = kg * 8 + c;
    cd val = C(0.0);
    if (valid && k < n) {
      val = y[((size_t)q * nrhs + ridx) * n + k];
      if (neg && ((k & 3) == 1 || (k & 3) == 2)) val = -val;   // D_c
    }
    digits(val.x * inv, dre[c]);
    digits(val.y * inv, dim_[c]);
  }
  const int jt = g / jtw, jj = g % jtw, nkt = npad / OZ_KT;
  const int kt = (kg * 8) / OZ_KT, kk = (kg * 8) % OZ_KT;
  const int ytile = oz_ytile(jtw);
  __nv_bfloat16* blk = Ysl + (((size_t)m * njt + jt) * nkt + kt) * oz_yblock(jtw);
  const int off = core_off(jj, kk);
#pragma unroll
  for (int s = 0; s < OZ_S; ++s) {
    __align__(16) __nv_bfloat16 re[8], im[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) { re[c] = __float2bfloat16(dre[c][s]); im[c] = __float2bfloat16(dim_[c][s]); }
    *(uint4*)(blk + (0 * OZ_S + s) * ytile + off) = *(uint4*)re;
    *(uint4*)(blk + (1 * OZ_S + s) * ytile + off) = *(uint4*)im;
  }
}

__device__ __forceinline__ void atomic_max_pos_oz(double* addr, double v) {
  atomicMax((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}

// CTA per (row tile, mode, job tile of JT columns); 128 threads; thread 0 issues copies and MMAs.
template <int JT>
__global__ void __launch_bounds__(128, 1)
    oz_residual_kernel(const __nv_bfloat16* __restrict__ Asl, const double* __restrict__ rowscale,
                       const __nv_bfloat16* __restrict__ Ysl, const double* __restrict__ colscale, int n, int npad,
                       int M, int nrhs, int njt, const cd* __restrict__ bw, cd* __restrict__ r,
                       double* __restrict__ rnorm, int* __restrict__ err) {
  constexpr int YT = oz_ytile(JT), YB = oz_yblock(JT);
  constexpr uint32_t TMEM_COLS = 2 * OZ_S * JT;   // 8 levels x re/im x JT columns
  extern __shared__ __align__(1024) unsigned char smem[];
  __nv_bfloat16* bufA = (__nv_bfloat16*)smem;                         // [2][OZ_ABLOCK]
  __nv_bfloat16* bufY = bufA + 2 * OZ_ABLOCK;                         // [2][YB]
  __shared__ __align__(8) uint64_t full[2], empty[2], drain;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  const int rt = blockIdx.x, m = blockIdx.y, jt = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nrt = npad / OZ_RT, nkt = npad / OZ_KT;
  const __nv_bfloat16* Ab = Asl + ((size_t)m * nrt + rt) * nkt * OZ_ABLOCK;
  const __nv_bfloat16* Yb = Ysl + ((size_t)m * njt + jt) * nkt * YB;
  const uint32_t abytes = OZ_ABLOCK * 2, ybytes = YB * 2;
  if (warp == 0) tc::tmem_alloc(&tmem_base, TMEM_COLS);
  if (tid == 0) {
    s_fail = 0;
    tc::mbar_init(&full[0], 1); tc::mbar_init(&full[1], 1);
    tc::mbar_init(&empty[0], 1); tc::mbar_init(&empty[1], 1);
    tc::mbar_init(&drain, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  auto load = [&](int kt) {
    int b = kt & 1;
    tc::mbar_expect_tx(&full[b], abytes + ybytes);
    tc::bulk_g2s(bufA + b * OZ_ABLOCK, Ab + (size_t)kt * OZ_ABLOCK, abytes, &full[b]);
    tc::bulk_g2s(bufY + b * YB, Yb + (size_t)kt * YB, ybytes, &full[b]);
  };
  if (tid == 0) {
    load(0);
    if (nkt > 1) load(1);
  }
  const uint32_t id_pos = tc::idesc_bf16_f32(OZ_RT, JT, false);
  const uint32_t id_neg = tc::idesc_bf16_f32(OZ_RT, JT, true);
  double zre[JT], zim[JT];
#pragma unroll
  for (int j = 0; j < JT; ++j) { zre[j] = 0.0; zim[j] = 0.0; }
  const int nchunk = (nkt + OZ_CHUNK - 1) / OZ_CHUNK;
  for (int c = 0; c < nchunk; ++c) {
    const int kt0 = c * OZ_CHUNK, kt1 = min(nkt, kt0 + OZ_CHUNK);
    if (tid == 0 && !s_fail) {
      for (int kt = kt0; kt < kt1; ++kt) {
        const int b = kt & 1;
        if (!tc::mbar_wait(&full[b], (kt >> 1) & 1)) { s_fail = 1; break; }
        tc::fence_after();
        // descriptors of slice 0 of this buffer; slice tiles follow at fixed
        // offsets (4 KiB for A, 1 KiB for y: 256 and 64 in the 16-byte units
        // of the descriptor's start-address field, which cannot carry)
        const uint64_t a_re0 = tc::desc_noswizzle(tc::smem_u32(bufA + b * OZ_ABLOCK), 128, 256);
        const uint64_t y_re0 = tc::desc_noswizzle(tc::smem_u32(bufY + b * YB), 128, 256);
        const uint64_t a_im0 = a_re0 + (uint64_t)(OZ_S * OZ_ATILE * 2 / 16);
        const uint64_t y_im0 = y_re0 + (uint64_t)(OZ_S * YT * 2 / 16);
        const uint32_t first = (kt == kt0) ? 1u : 0u;
#pragma unroll
        for (int s = 0; s < OZ_S; ++s) {
#pragma unroll
          for (int t = 0; t < OZ_S - s; ++t) {
            const int l = s + t;
            const uint32_t acc_re = tmem + (uint32_t)((l * 2 + 0) * JT);
            const uint32_t acc_im = tmem + (uint32_t)((l * 2 + 1) * JT);
            const uint64_t are = a_re0 + (uint64_t)(s * (OZ_ATILE * 2 / 16));
            const uint64_t aim = a_im0 + (uint64_t)(s * (OZ_ATILE * 2 / 16));
            const uint64_t yre = y_re0 + (uint64_t)(t * (YT * 2 / 16));
            const uint64_t yim = y_im0 + (uint64_t)(t * (YT * 2 / 16));
            const uint32_t fresh = (s == 0) ? (first ^ 1u) : 1u;  // first product of this level in the chunk
            tc::mma_bf16(acc_re, are, yre, id_pos, fresh);
            tc::mma_bf16(acc_re, aim, yim, id_neg, 1u);
            tc::mma_bf16(acc_im, are, yim, id_pos, fresh);
            tc::mma_bf16(acc_im, aim, yre, id_pos, 1u);
          }
        }
        tc::commit(&empty[b]);
        // refill the buffer of the previous k-tile with k-tile kt + 1
        if (kt >= 1 && kt + 1 < nkt) {
          const int pb = (kt - 1) & 1;
          if (!tc::mbar_wait(&empty[pb], ((kt - 1) >> 1) & 1)) { s_fail = 1; break; }
          load(kt + 1);
        }
      }
      tc::commit(&drain);
    }
    __syncthreads();
    if (s_fail) break;
    if (!tc::mbar_wait(&drain, c & 1)) { atomicExch(&s_fail, 1); }
    __syncthreads();
    if (s_fail) break;
    tc::fence_after();
    // drain: this warp's 32 rows, all levels
    const uint32_t tw = tmem + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
    for (int l = 0; l < OZ_S; ++l) {
      const double sc = ldexp(1.0, -7 * (l + 2));
      float v[JT];
      tc::tmem_ld32(tw + (uint32_t)((l * 2 + 0) * JT), v);
#pragma unroll
      for (int j = 0; j < JT; ++j) zre[j] = fma(sc, (double)v[j], zre[j]);
      tc::tmem_ld32(tw + (uint32_t)((l * 2 + 1) * JT), v);
#pragma unroll
      for (int j = 0; j < JT; ++j) zim[j] = fma(sc, (double)v[j], zim[j]);
    }
    tc::fence_before();
    __syncthreads();
    tc::fence_after();
  }
  if (s_fail) {
    if (tid == 0) {
      atomicExch(err, 1);
      // let copies still in flight land before the CTA exits (bounded)
      tc::mbar_wait(&full[0], 0, 1 << 20);
      tc::mbar_wait(&full[1], 0, 1 << 20);
    }
  } else {
    const int i = rt * OZ_RT + warp * 32 + lane;
    if (i < n) {
      const double si = rowscale[(size_t)m * npad + i];
#pragma unroll 1
      for (int j = 0; j < JT; ++j) {
        const int g = jt * JT + j;
        int q, ridx;
        bool neg;
        if (!job_vec(m, M, nrhs, g, &q, &ridx, &neg)) continue;
        const double sc = si * colscale[(size_t)m * njt * JT + g];
        cd z = C(sc * zre[j], sc * zim[j]);
        if (neg && ((i & 3) == 0 || (i & 3) == 3)) z = -z;   // D_r
        const size_t idx = ((size_t)q * nrhs + ridx) * n + i;
        cd val = bw[idx] - z;
        r[idx] = val;
        atomic_max_pos_oz(rnorm + (size_t)q * nrhs + ridx, cabs(val));
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  if (warp == 0) tc::tmem_dealloc(tmem, TMEM_COLS);
}

template <int JT>
static void oz_residual_launch(const __nv_bfloat16* Asl, const double* rowscale, int n, int npad, int M,
                               const cd* bw, cd* r, int nrhs, int njt, double* rnorm, const __nv_bfloat16* Ysl,
                               const double* colscale, int* err, cudaStream_t s) {
  const int smem = 2 * (OZ_ABLOCK + oz_yblock(JT)) * 2;
  cudaFuncSetAttribute(oz_residual_kernel<JT>, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  oz_residual_kernel<JT><<<dim3(npad / OZ_RT, M + 1, njt), 128, smem, s>>>(Asl, rowscale, Ysl, colscale, n, npad,
                                                                           M, nrhs, njt, bw, r, rnorm, err);
}

void ozaki_residual(const __nv_bfloat16* Asl, const double* rowscale, int n, int npad, int M, const cd* bw,
                    const cd* y, cd* r, int nrhs, double* rnorm, __nv_bfloat16* Ysl, double* colscale, int* err,
                    cudaStream_t s) {
  const int jt = ozaki_job_tile(nrhs), njt = ozaki_job_tiles(nrhs);
  oz_colscale_kernel<<<dim3(njt * jt, M + 1), 256, 0, s>>>(y, n, M, nrhs, njt, jt, colscale);
  const int threads = njt * jt * (npad / 8);
  oz_slice_vectors_kernel<<<dim3((threads + 127) / 128, M + 1), 128, 0, s>>>(y, n, npad, M, nrhs, njt, jt, colscale,
                                                                           Ysl);
  cudaMemsetAsync(rnorm, 0, sizeof(double) * (2 * M + 1) * nrhs, s);
  if (jt == 16) oz_residual_launch<16>(Asl, rowscale, n, npad, M, bw, r, nrhs, njt, rnorm, Ysl, colscale, err, s);
  else oz_residual_launch<OZ_JT>(Asl, rowscale, n, npad, M, bw, r, nrhs, njt, rnorm, Ysl, colscale, err, s);
}
