// Interfaces of the tcgen05 GEMMs (see umma3.cu and umma_bf16.cu).
#pragma once

#include <cuda.h>

#include "common.cuh"

namespace rlu {

// FP32-accurate tensor-core products from exact TF32 splits (see umma3.cu).
enum { U3_MODE_Y2 = 0, U3_MODE_C3 = 1, U3_MODE_G3 = 2, U3_MODE_Y3 = 3 };

struct Umma3Args {
  float* out;
  int64_t ldo;
  size_t split_stride;
  int M, N, K, BN, kchunk, stages;
  int ntiles;  // N tiles; grid x = row tiles x N tiles, the N tile varying fastest
  int bn_last;  // MMA width of the last N tile (BF16 kernels)
  bool out_colmajor;
  int32_t* status;
  // sub_pos != nullptr: out -= D instead of out = D, only in the rows r whose
  // sub_pos[r] >= sub_min (one-tile kernel, column-major out, no split-K)
  const int32_t* sub_pos;
  int sub_min;
};

// Y2: A0 = A (M x K row-major, lda), B0 = G^T (N x K row-major, ldb).
// C3: A0 = A stored K x M row-major (lda), B0/B1 = hi/lo of B (N x K row-major, ldb).
// G3: A0/A1 = hi/lo of A (M x K, lda), B0/B1 = hi/lo of B (N x K, ldb).
// Y3: A0 = A (M x K row-major, split on chip), B0/B1 = hi/lo of B (N x K row-major, ldb).
// out == nullptr: only the row-major FP32 partial slices (splits x M x N) are written.
struct Umma3Op {
  const float* A0;
  const float* A1;
  int64_t lda;
  const float* B0;
  const float* B1;
  int64_t ldb;
  int64_t M, N, K;
  float* out;
  int64_t ldo;
  bool out_colmajor;
  int splits;
  float* partial;
  int32_t* status;
  const int32_t* sub_pos;  // see Umma3Args
  int sub_min;
};

int32_t umma3_gemm(int mode, const Umma3Op& op, cudaStream_t s);

// Rank-w (w <= 96) trailing update of a pivoted LU on the tensor cores, FP32-accurate (three
// TF32 products): X[r][c] -= sum_s X[r][p0 + s] U[s][c] for the columns c_begin <= c < c_end
// of every row r whose position posg[r] >= p0 + w. X column-major (R x C, ldx, ldx % 4 == 0,
// 16-byte aligned), U = the solved pivot rows (u12 + s * ldu, absolute column index), bt
// scratch of 2 x 96 x (c_end - c_begin) floats (U^T's TF32 parts). RLU_EUNSUPPORTED when
// the shapes or alignments do not suit it (the caller then runs the SIMT update).
int32_t umma3_trail(float* X, int64_t ldx, int R, int c_begin, int c_end, int p0, int w,
                    const int32_t* posg, const float* u12, int64_t ldu, float* bt,
                    int32_t* status, cudaStream_t s);

// Batched form (Y2 and C3 only, N <= 256, whole K per CTA): one record per problem with its
// tensor maps (A0, A1, B0, B1) and arguments, in device memory, 64-byte aligned.
struct U3Job {
  CUtensorMap map[4];
  Umma3Args a;
};
// Fills job (host memory) for op; *stage_bytes = its shared-memory slot size. ta: the slot
// of the kernel that keeps A's TF32 parts in tensor memory (umma3_batched with ta).
int32_t umma3_make_job(int mode, const Umma3Op& op, U3Job* job, int* stage_bytes,
                       bool ta = false);
// Ring slots (at most 4) of this slot size that fit one CTA, or that still let ctas_per_sm
// CTAs share an SM's shared memory (each CTA holds 256 of an SM's 512 TMEM columns).
int32_t umma3_stages_for(int stage_bytes, int ctas_per_sm = 1);
// One launch over a tile list (device, ntiles entries of (record, 128-row tile)), modes Y2
// and C3, every record's BN <= 128: persistent CTAs (as many as stay resident) take tiles
// from the list through counter (device, zeroed on s before the launch) and run one ring of
// k-steps across their tiles with a double-buffered TMEM accumulator. ta: one CTA per SM,
// A's TF32 parts in tensor memory (the MMAs read A from TMEM); else the parts go through
// shared memory and two CTAs may share an SM.
int32_t umma3_batched(int mode, const U3Job* jobs_dev, const int2* tiles_dev, int ntiles,
                      int stages, int max_stage_bytes, unsigned* counter, cudaStream_t s,
                      bool ta = false);

// BF16 products (see umma_bf16.cu), same output conventions as Umma3Op.
// Y : A (M x K row-major BF16, lda), B0 = G^T (N x K row-major BF16, ldb), one product.
// C3: D = sum over the parts of B_p A: A stored K x N row-major BF16 (lda); B0/B1/B2 =
//     hi/mid/lo BF16 parts of the M x K left factor (K contiguous, ldb).
// Y3: A as for Y; B0/B1/B2 = hi/mid/lo BF16 parts of the N x K right factor (ldb).
enum { UB_MODE_Y = 0, UB_MODE_C3 = 1, UB_MODE_Y3 = 2 };
struct UmmaBf16Op {
  const void* A;
  int64_t lda;
  const void* B0;
  const void* B1;
  const void* B2;
  int64_t ldb;
  int64_t M, N, K;
  float* out;
  int64_t ldo;
  bool out_colmajor;
  int splits;
  float* partial;
  int32_t* status;
};
int32_t umma_bf16_gemm(int mode, const UmmaBf16Op& op, cudaStream_t s);
// FP8 e4m3 projection with per-tile power-of-two scales (see umma_fp8.cu).
// A8: M x K e4m3 (lda8 bytes per row, K zero-padded to a multiple of 128), SA: one UE8M0
// byte per row and 128-column block (lds per row); G8: N x K e4m3 (row j = column j of G,
// ldg8 bytes), SG: one byte per 128 x 128 block (lsg per K block). out = A8 G8^T, FP32.
struct Fp8Op {
  const uint8_t* A8;
  int64_t lda8;
  const uint8_t* SA;
  int64_t lds;
  const uint8_t* G8;
  int64_t ldg8;
  const uint8_t* SG;
  int64_t lsg;
  int64_t M, N, K;
  float* out;
  int64_t ldo;
  bool out_colmajor;
  int splits;
  float* partial;
  int32_t* status;
};
int64_t fp8_ld(int64_t K);  // bytes per row of an e4m3 operand with K columns
int32_t fp8_quantize_a(const void* A, int64_t lda, int64_t M, int64_t K, uint8_t* A8,
                       int64_t ld8, uint8_t* SA, int64_t lds, cudaStream_t s);
int32_t fp8_quantize_g(const float* G, int64_t ldg, int64_t K, int64_t N, uint8_t* G8,
                       int64_t ld8, uint8_t* SG, int64_t lsg, cudaStream_t s);
int32_t umma_fp8_y(const Fp8Op& op, cudaStream_t s);
int umma_fp8_splits(int64_t M, int64_t K, int64_t N);

// split-K factor that fills the SMs for an M x N output (N tiles of bn columns)
int umma_bf16_splits(int64_t M, int64_t K, int64_t N, int bn);
int umma3_splits(int64_t M, int64_t K, int64_t N);

// Fixed-order sum of row-major FP32 partial slices into out (row- or column-major).
int32_t splitk_reduce_f32(const float* part, int splits, int64_t M, int64_t N, float* out,
                          int64_t ldo, bool out_rowmajor, cudaStream_t s);

// Fixed-order sum of column-major FP32 partial slices (M x N, ld M each, slice stride M N)
// into a column-major output (ldo).
int32_t splitk_reduce_cm_f32(const float* part, int splits, int64_t M, int64_t N, float* out,
                             int64_t ldo, cudaStream_t s);

// Fixed-order FP64 sum of row-major FP32 partial slices into a row-major FP64 matrix.
int32_t splitk_reduce_f64(const float* part, int splits, int64_t M, int64_t N, double* out,
                          int64_t ldo, cudaStream_t s);

}  // namespace rlu
