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
// accumulator per level, [Re | Im] side by side (8 x 2 jt columns, jt the job
// tile of 16 or 32 right-hand-side columns); every 256 values of k they are
// drained into FP64 registers.  The complex product takes two MMAs per digit
// pair: the B operand stacks the digits of Re y over those of Im y (2 jt
// rows), so Re a [Re y | Im y] + Im a [-Im y | Re y] lands in [Re | Im] of the
// accumulator; the y slices are stored as [-Im, Re, Im] per digit, and the
// two B operands start at Re and at -Im.
// Operand tiles are stored in global memory in the shared-memory layout of the
// MMA (no-swizzle K-major core matrices), so each 16-wide k-tile is a single
// bulk asynchronous copy (TMA).  The residual kernel is warp-specialised: a
// copy thread keeps a ring of k-tile stages full, an MMA thread consumes
// them, and four drain warps empty the accumulators of a finished 256-k
// chunk while the MMAs of the next chunk run (two accumulator sets in tensor
// memory where they fit).
#include <algorithm>
#include <cstdio>
#include "ozaki.cuh"
#include "digits.cuh"
#include "tc.cuh"

#define OZ_ATILE (OZ_RT * OZ_KT)          // bf16 elements per slice tile of A
#define OZ_ABLOCK (2 * OZ_S * OZ_ATILE)   // per (row tile, k-tile): re/im x 8 slices
// slice tile and block of Y for a job tile of jt right-hand-side columns
__host__ __device__ constexpr int oz_ytile(int jt) { return jt * OZ_KT; }
__host__ __device__ constexpr int oz_yblock(int jt) { return 3 * OZ_S * jt * OZ_KT; }  // [digit][-Im, Re, Im]

size_t ozaki_matrix_slices_elems(int npad, int batch) {
  return (size_t)batch * (npad / OZ_RT) * (npad / OZ_KT) * OZ_ABLOCK;
}
size_t ozaki_vector_slices_elems(int npad, int batch, int njt, int jt) {
  return (size_t)batch * njt * (npad / OZ_KT) * oz_yblock(jt);
}

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

// thread per (row i, group of 8 consecutive k): 16 digit rows of 16 bytes.
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
    __align__(16) __nv_bfloat16 re[8], im[8], nim[8];
#pragma unroll
    for (int c = 0; c < 8; ++c) {
      re[c] = __float2bfloat16(dre[c][s]);
      im[c] = __float2bfloat16(dim_[c][s]);
      nim[c] = __float2bfloat16(-dim_[c][s]);
    }
    *(uint4*)(blk + (3 * s + 0) * ytile + off) = *(uint4*)nim;
    *(uint4*)(blk + (3 * s + 1) * ytile + off) = *(uint4*)re;
    *(uint4*)(blk + (3 * s + 2) * ytile + off) = *(uint4*)im;
  }
}

__device__ __forceinline__ void atomic_max_pos_oz(double* addr, double v) {
  atomicMax((unsigned long long*)addr, (unsigned long long)__double_as_longlong(v));
}

// Shape of the residual kernel for a job tile of JT columns.
template <int JT> struct OzShape {
  static constexpr int YT = oz_ytile(JT), YB = oz_yblock(JT);
  static constexpr uint32_t SET_COLS = 2 * OZ_S * JT;          // accumulators of one chunk: 8 levels x [Re | Im]
  static constexpr int NACC = (2 * SET_COLS <= 512) ? 2 : 1;   // two sets (drain overlaps the next chunk) if they fit
  static constexpr uint32_t TMEM_COLS = 512;                   // NACC x SET_COLS, allocated as a power of two
  static constexpr int STAGE = (OZ_ABLOCK + YB) * 2;           // bytes of one k-tile (A and y digits)
  static constexpr int NST = 2;                                // k-tile stages in shared memory
  static constexpr int SMEM = NST * STAGE;
  static constexpr int THREADS = 192;                          // warps 0-3 drain, 4 copies, 5 issues MMAs
};
static_assert(OzShape<16>::NACC * OzShape<16>::SET_COLS <= 512 && OzShape<OZ_JT>::NACC * OzShape<OZ_JT>::SET_COLS <= 512,
              "accumulator sets exceed tensor memory");
static_assert(OzShape<OZ_JT>::SMEM <= 227 * 1024, "stages exceed shared memory");

// CTA per (row tile, mode, job tile of JT columns).  Every wait is bounded:
// a role that gives up sets the CTA's failure flag (and *err), the others
// stop at their next wait, and before the CTA exits the copy thread lets its
// copies in flight land and the MMA thread waits for its MMAs.
template <int JT>
__global__ void __launch_bounds__(192, 1)
    oz_residual_kernel(const __nv_bfloat16* __restrict__ Asl, const double* __restrict__ rowscale,
                       const __nv_bfloat16* __restrict__ Ysl, const double* __restrict__ colscale, int n, int npad,
                       int M, int nrhs, int njt, const cd* __restrict__ bw, cd* __restrict__ r,
                       double* __restrict__ rnorm, int* __restrict__ err) {
  using S = OzShape<JT>;
  constexpr int NST = S::NST, NACC = S::NACC;
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[NST], empty[NST], tfull[NACC], tempty[NACC], mdone;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  volatile int* fail = &s_fail;
  const int rt = blockIdx.x, m = blockIdx.y, jt = blockIdx.z;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  const int nrt = npad / OZ_RT, nkt = npad / OZ_KT;
  const int nchunk = (nkt + OZ_CHUNK - 1) / OZ_CHUNK;
  if (warp == 0) tc::tmem_alloc(&tmem_base, S::TMEM_COLS);
  if (tid == 32) {
    s_fail = 0;
#pragma unroll
    for (int b = 0; b < NST; ++b) { tc::mbar_init(&full[b], 1); tc::mbar_init(&empty[b], 1); }
#pragma unroll
    for (int b = 0; b < NACC; ++b) { tc::mbar_init(&tfull[b], 1); tc::mbar_init(&tempty[b], 4); }
    tc::mbar_init(&mdone, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  double zre[JT], zim[JT];
#pragma unroll
  for (int j = 0; j < JT; ++j) { zre[j] = 0.0; zim[j] = 0.0; }
  int issued = 0;  // copy thread: k-tiles whose copies were issued
  if (warp == 4) {
    if (lane == 0) {
      const __nv_bfloat16* Ab = Asl + ((size_t)m * nrt + rt) * nkt * OZ_ABLOCK;
      const __nv_bfloat16* Yb = Ysl + ((size_t)m * njt + jt) * nkt * S::YB;
      for (int kt = 0; kt < nkt; ++kt) {
        const int st = kt % NST;
        if (kt >= NST && !tc::mbar_wait(&empty[st], ((kt / NST) - 1) & 1)) { *fail = 1; break; }
        if (*fail) break;
        unsigned char* base = smem + (size_t)st * S::STAGE;
        tc::mbar_expect_tx(&full[st], S::STAGE);
        tc::bulk_g2s(base, Ab + (size_t)kt * OZ_ABLOCK, OZ_ABLOCK * 2, &full[st]);
        tc::bulk_g2s(base + OZ_ABLOCK * 2, Yb + (size_t)kt * S::YB, S::YB * 2, &full[st]);
        issued = kt + 1;
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(OZ_RT, 2 * JT, false);
      int kt = 0;
      for (int c = 0; c < nchunk && !*fail; ++c) {
        const int set = c % NACC;
        if (c >= NACC && !tc::mbar_wait(&tempty[set], ((c / NACC) - 1) & 1)) { *fail = 1; break; }
        tc::fence_after();
        const uint32_t acc0 = tmem + (uint32_t)set * S::SET_COLS;
        const int kt1 = min(nkt, (c + 1) * OZ_CHUNK);
        for (; kt < kt1; ++kt) {
          const int st = kt % NST;
          if (!tc::mbar_wait(&full[st], (kt / NST) & 1)) { *fail = 1; break; }
          tc::fence_after();
          unsigned char* base = smem + (size_t)st * S::STAGE;
          // digit s of Re a at s tiles, of Im a at OZ_S + s tiles (4 KiB each);
          // digit t of y: [-Im, Re, Im] at 3t tiles (JT x 16 each)
          const uint64_t a0 = tc::desc_noswizzle(tc::smem_u32(base), 128, 256);
          const uint64_t y0 = tc::desc_noswizzle(tc::smem_u32(base + OZ_ABLOCK * 2), 128, 256);
          const bool first = kt == c * OZ_CHUNK;
#pragma unroll
          for (int s = 0; s < OZ_S; ++s) {
#pragma unroll
            for (int t = 0; t < OZ_S - s; ++t) {
              const uint32_t acc = acc0 + (uint32_t)((s + t) * 2 * JT);
              const uint64_t are = a0 + (uint64_t)(s * (OZ_ATILE * 2 / 16));
              const uint64_t aim = a0 + (uint64_t)((OZ_S + s) * (OZ_ATILE * 2 / 16));
              const uint64_t yri = y0 + (uint64_t)((3 * t + 1) * (S::YT * 2 / 16));  // [Re | Im]
              const uint64_t ymr = y0 + (uint64_t)((3 * t + 0) * (S::YT * 2 / 16));  // [-Im | Re]
              tc::mma_bf16(acc, are, yri, idesc, (first && s == 0) ? 0u : 1u);
              tc::mma_bf16(acc, aim, ymr, idesc, 1u);
            }
          }
          tc::commit(&empty[st]);  // the stage is free once these MMAs have read it
        }
        if (*fail) break;
        tc::commit(&tfull[set]);   // the chunk's accumulators are complete
      }
      tc::commit(&mdone);          // arrives once every MMA issued above has completed
      if (!tc::mbar_wait(&mdone, 0)) *fail = 1;
    }
  } else {
    // drain warps: warp w owns tensor-memory lanes (rows) 32w .. 32w + 31
    for (int c = 0; c < nchunk; ++c) {
      const int set = c % NACC;
      if (!tc::mbar_wait(&tfull[set], (c / NACC) & 1)) { *fail = 1; break; }
      tc::fence_after();
      const uint32_t tw = tmem + (uint32_t)set * S::SET_COLS + ((uint32_t)(warp * 32) << 16);
#pragma unroll 1
      for (int l = 0; l < OZ_S; ++l) {
        const double sc = ldexp(1.0, -7 * (l + 2));
#pragma unroll
        for (int h = 0; h < 2 * JT; h += 32) {  // 32 columns per load: [Re | Im] of JT = 16, half of it for JT = 32
          float v[32];
          tc::tmem_ld32(tw + (uint32_t)(l * 2 * JT + h), v);
#pragma unroll
          for (int u = 0; u < 32; ++u) {
            const int col = h + u;
            if (col < JT) zre[col] = fma(sc, (double)v[u], zre[col]);
            else zim[col - JT] = fma(sc, (double)v[u], zim[col - JT]);
          }
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[set]);
    }
  }
  __syncthreads();
  if (*fail) {
    if (tid == 0) atomicExch(err, 1);
    if (warp == 4 && lane == 0) {
      // let the copies still in flight land before the CTA exits (bounded):
      // the newest copy of each stage completes the newest phase of its barrier
      for (int st = 0; st < NST; ++st) {
        const int last = issued - 1 - ((issued - 1 - st) % NST + NST) % NST;  // newest k-tile issued into st
        if (last >= 0 && last < issued) tc::mbar_wait(&full[st], (last / NST) & 1, 1 << 20);
      }
    }
  } else if (warp < 4) {
    const int i = rt * OZ_RT + warp * 32 + lane;
    if (i < n) {
      const double si = rowscale[(size_t)m * npad + i];
#pragma unroll
      for (int j = 0; j < JT; ++j) {  // unrolled: zre / zim stay in registers
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
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, S::TMEM_COLS);
}

template <int JT>
static void oz_residual_launch(const __nv_bfloat16* Asl, const double* rowscale, int n, int npad, int M,
                               const cd* bw, cd* r, int nrhs, int njt, double* rnorm, const __nv_bfloat16* Ysl,
                               const double* colscale, int* err, cudaStream_t s) {
  using S = OzShape<JT>;
  cudaFuncSetAttribute(oz_residual_kernel<JT>, cudaFuncAttributeMaxDynamicSharedMemorySize, S::SMEM);
  oz_residual_kernel<JT><<<dim3(npad / OZ_RT, M + 1, njt), S::THREADS, S::SMEM, s>>>(
      Asl, rowscale, Ysl, colscale, n, npad, M, nrhs, njt, bw, r, rnorm, err);
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

// ---------------------------------------------------------------------------
// Real product Y = A B with A given by the digits of its rows (row scales
// Ascale, a power of two each) and B by the digits of its columns (one scale
// bscale): Y[c * ldy + r] for the first ncols columns.  Operand blocks per
// (row tile, k-tile) and (column tile, k-tile) hold the 8 digits of a 128 x 16
// (32 x 16) tile in the MMA's layout.  K is at most OZR_KMAX, so that every
// level's sum stays an exact FP32 integer (8 digit pairs x 272 x 64^2 < 2^24)
// and one drain per tile suffices; the levels are joined exactly in 64-bit
// integers (levels 0-3 and 4-7 apart) and converted to FP64 twice per entry.
// Persistent: CTA b takes tiles b, b + gridDim.x, ... (column tile fastest,
// so the CTAs of one row tile share its A in L2); warps 0-3 drain, 4 copies
// through a ring of k-tile stages, 5 issues MMAs into one of two accumulator
// sets (8 levels x 32 columns each), so a tile's drain overlaps the next
// tile's products.
#define OZR_NT 32
#define OZR_BBLOCK (OZ_S * OZR_NT * OZ_KT)       // bf16 elements per (column tile, k-tile)
#define OZR_ABLOCK (OZ_S * OZ_ATILE)             // per (row tile, k-tile)
#define OZR_STAGE ((OZR_ABLOCK + OZR_BBLOCK) * 2)
#define OZR_NST 4
#define OZR_SET (OZ_S * OZR_NT)                  // tensor-memory columns of one accumulator set

__global__ void __launch_bounds__(192, 1)
    oz_real_gemm_kernel(const __nv_bfloat16* __restrict__ Asl, const double* __restrict__ Ascale,
                        const __nv_bfloat16* __restrict__ Bsl, double bscale, int nkt, int ntc, long long ntiles,
                        double* __restrict__ Y, int ldy, int ncols, int* __restrict__ err) {
  extern __shared__ __align__(1024) unsigned char smem[];
  __shared__ __align__(8) uint64_t full[OZR_NST], empty[OZR_NST], tfull[2], tempty[2], mdone;
  __shared__ uint32_t tmem_base;
  __shared__ int s_fail;
  volatile int* fail = &s_fail;
  const int tid = threadIdx.x, warp = tid >> 5, lane = tid & 31;
  if (warp == 0) tc::tmem_alloc(&tmem_base, 512);
  if (tid == 32) {
    s_fail = 0;
#pragma unroll
    for (int b = 0; b < OZR_NST; ++b) { tc::mbar_init(&full[b], 1); tc::mbar_init(&empty[b], 1); }
    for (int b = 0; b < 2; ++b) { tc::mbar_init(&tfull[b], 1); tc::mbar_init(&tempty[b], 4); }
    tc::mbar_init(&mdone, 1);
    tc::mbar_fence_init();
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  const uint32_t tmem = tmem_base;
  int issued = 0;
  if (warp == 4) {
    if (lane == 0) {
      int q = 0;
      for (long long t = blockIdx.x; t < ntiles && !*fail; t += gridDim.x) {
        const int nt = (int)(t % ntc);
        const long long rt = t / ntc;
        const __nv_bfloat16* Ab = Asl + (size_t)rt * nkt * OZR_ABLOCK;
        const __nv_bfloat16* Bb = Bsl + (size_t)nt * nkt * OZR_BBLOCK;
        for (int kt = 0; kt < nkt; ++kt, ++q) {
          const int st = q % OZR_NST;
          if (q >= OZR_NST && !tc::mbar_wait(&empty[st], ((q / OZR_NST) - 1) & 1)) { *fail = 1; break; }
          unsigned char* base = smem + (size_t)st * OZR_STAGE;
          tc::mbar_expect_tx(&full[st], OZR_STAGE);
          tc::bulk_g2s(base, Ab + (size_t)kt * OZR_ABLOCK, OZR_ABLOCK * 2, &full[st]);
          tc::bulk_g2s(base + OZR_ABLOCK * 2, Bb + (size_t)kt * OZR_BBLOCK, OZR_BBLOCK * 2, &full[st]);
          issued = q + 1;
        }
      }
    }
  } else if (warp == 5) {
    if (lane == 0) {
      const uint32_t idesc = tc::idesc_bf16_f32(OZ_RT, OZR_NT, false);
      int q = 0, k = 0;
      for (long long t = blockIdx.x; t < ntiles && !*fail; t += gridDim.x, ++k) {
        const int set = k & 1;
        if (k >= 2 && !tc::mbar_wait(&tempty[set], ((k >> 1) - 1) & 1)) { *fail = 1; break; }
        tc::fence_after();
        const uint32_t acc0 = tmem + (uint32_t)(set * OZR_SET);
        for (int kt = 0; kt < nkt; ++kt, ++q) {
          const int st = q % OZR_NST;
          if (!tc::mbar_wait(&full[st], (q / OZR_NST) & 1)) { *fail = 1; break; }
          tc::fence_after();
          unsigned char* base = smem + (size_t)st * OZR_STAGE;
          const uint64_t a0 = tc::desc_noswizzle(tc::smem_u32(base), 128, 256);
          const uint64_t b0 = tc::desc_noswizzle(tc::smem_u32(base + OZR_ABLOCK * 2), 128, 256);
#pragma unroll
          for (int s = 0; s < OZ_S; ++s) {
#pragma unroll
            for (int u = 0; u < OZ_S - s; ++u) {
              const uint32_t acc = acc0 + (uint32_t)((s + u) * OZR_NT);
              const uint64_t ad = a0 + (uint64_t)(s * (OZ_ATILE * 2 / 16));
              const uint64_t bd = b0 + (uint64_t)(u * (OZR_NT * OZ_KT * 2 / 16));
              tc::mma_bf16(acc, ad, bd, idesc, (kt == 0 && s == 0) ? 0u : 1u);  // (0, u) opens level u
            }
          }
          tc::commit(&empty[st]);
        }
        if (*fail) break;
        tc::commit(&tfull[set]);
      }
      tc::commit(&mdone);  // arrives once every MMA issued above has completed
      if (!tc::mbar_wait(&mdone, 0)) *fail = 1;
    }
  } else {
    // drain: this warp's 32 rows, 16 columns at a time, levels joined in integers
    int k = 0;
    for (long long t = blockIdx.x; t < ntiles; t += gridDim.x, ++k) {
      const int set = k & 1;
      if (!tc::mbar_wait(&tfull[set], (k >> 1) & 1)) { *fail = 1; break; }
      tc::fence_after();
      const int nt = (int)(t % ntc);
      const long long rt = t / ntc;
      const long long r = rt * OZ_RT + warp * 32 + lane;
      const double sc = Ascale[r] * bscale;
      const uint32_t tw = tmem + (uint32_t)(set * OZR_SET) + ((uint32_t)(warp * 32) << 16);
#pragma unroll
      for (int c0 = 0; c0 < OZR_NT; c0 += 16) {
        long long hi[16], lo[16];
#pragma unroll
        for (int c = 0; c < 16; ++c) { hi[c] = 0; lo[c] = 0; }
#pragma unroll
        for (int l = 0; l < OZ_S; ++l) {
          float v[16];
          tc::tmem_ld16(tw + (uint32_t)(l * OZR_NT + c0), v);
#pragma unroll
          for (int c = 0; c < 16; ++c) {
            const long long iv = (long long)__float2int_rn(v[c]);  // an exact integer below 2^24
            if (l < 4) hi[c] = hi[c] * 128 + iv;
            else lo[c] = lo[c] * 128 + iv;
          }
        }
        // hi = sum_{l<4} acc_l 2^{7(3-l)}, lo = sum_{l>=4} acc_l 2^{7(7-l)};
        // level l carries 2^{-7(l+2)}: value = hi 2^-35 + lo 2^-63
#pragma unroll
        for (int c = 0; c < 16; ++c) {
          const int col = nt * OZR_NT + c0 + c;
          if (col < ncols)
            Y[(size_t)col * ldy + r] = sc * fma((double)hi[c], 2.9103830456733704e-11, (double)lo[c] * 1.0842021724855044e-19);
        }
      }
      tc::fence_before();
      __syncwarp();
      if (lane == 0) tc::mbar_arrive(&tempty[set]);
    }
  }
  __syncthreads();
  if (*fail) {
    if (tid == 0 && err) atomicExch(err, 1);
    if (warp == 4 && lane == 0) {
      for (int st = 0; st < OZR_NST; ++st) {
        const int last = issued - 1 - ((issued - 1 - st) % OZR_NST + OZR_NST) % OZR_NST;
        if (last >= 0) tc::mbar_wait(&full[st], (last / OZR_NST) & 1, 1 << 20);
      }
    }
  }
  tc::fence_before();
  __syncthreads();
  tc::fence_after();
  if (warp == 0) tc::tmem_dealloc(tmem, 512);
}

size_t ozaki_real_a_elems(int rows_pad, int nkt) { return (size_t)(rows_pad / OZ_RT) * nkt * OZR_ABLOCK; }
size_t ozaki_real_b_elems(int ncols, int nkt) { return (size_t)((ncols + OZR_NT - 1) / OZR_NT) * nkt * OZR_BBLOCK; }

void ozaki_real_gemm(const __nv_bfloat16* Asl, const double* Ascale, int rows_pad, const __nv_bfloat16* Bsl,
                     double bscale, int nkt, double* Y, int ldy, int ncols, int* err, cudaStream_t s) {
  const int smem = OZR_NST * OZR_STAGE;
  cudaFuncSetAttribute(oz_real_gemm_kernel, cudaFuncAttributeMaxDynamicSharedMemorySize, smem);
  const int ntc = (ncols + OZR_NT - 1) / OZR_NT;
  const long long ntiles = (long long)ntc * (rows_pad / OZ_RT);
  int dev = 0, sms = 152;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&sms, cudaDevAttrMultiProcessorCount, dev);
  const int grid = (int)std::min<long long>(ntiles, sms);
  oz_real_gemm_kernel<<<grid, 192, smem, s>>>(Asl, Ascale, Bsl, bscale, nkt, ntc, ntiles, Y, ldy, ncols, err);
}

// Digits of the columns of B[k][c] = b(k, c) / bscale for the real product
// (host): balanced base-128 digits of round(v 2^56), the same digits as on
// the device, in the operand layout of oz_real_gemm_kernel.
void ozaki_real_b_host(const double* b, int K, int ncols, double bscale, int nkt, __nv_bfloat16* out) {
  const int ntile = (ncols + OZR_NT - 1) / OZR_NT;
  for (size_t e = 0; e < (size_t)ntile * nkt * OZR_BBLOCK; ++e) out[e] = __float2bfloat16(0.f);
  for (int c = 0; c < ncols; ++c)
    for (int k = 0; k < K; ++k) {
      long long F = llrint(b[(size_t)k * ncols + c] / bscale * 72057594037927936.0);  // 2^56
      int d[OZ_S];
      for (int q = OZ_S - 1; q >= 1; --q) {
        const long long dd = ((F + 64) & 127) - 64;
        d[q] = (int)dd;
        F = (F - dd) >> 7;
      }
      d[0] = (int)F;
      const int t = c / OZR_NT, cc = c % OZR_NT, kt = k / OZ_KT, kk = k % OZ_KT;
      const int off = ((cc >> 3) * 2 + (kk >> 3)) * 64 + (cc & 7) * 8 + (kk & 7);
      for (int q = 0; q < OZ_S; ++q)
        out[((size_t)t * nkt + kt) * OZR_BBLOCK + (size_t)q * OZR_NT * OZ_KT + off] = __float2bfloat16((float)d[q]);
    }
}
