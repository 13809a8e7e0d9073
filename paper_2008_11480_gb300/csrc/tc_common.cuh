// Pieces shared by the one-CTA and the CTA-pair tensor-core GEMM kernels:
// work-item decoding and the fused epilogue of one accumulator tile.
#pragma once
#include "internal.h"
#include "ptx.cuh"

namespace nsgb {
namespace tc {

// Work item w of this CTA (cluster rank `rank` of CM along M): problem, tile
// row (in 128-row units) and tile column.
__device__ __forceinline__ void decode_item(const TcParams& p, int w, int rank, int CM, int& pi, int& mt, int& nt) {
  if (p.gprob != nullptr) {
    const TcItem it = p.items[w];
    pi = it.prob;
    mt = it.mt;
    nt = it.nt;
    return;
  }
  pi = 0;
#pragma unroll 1
  for (int i = 1; i < p.nprob; ++i)
    if (w >= p.prob[i].tile_begin) pi = i;
  const TcProblem& P = p.prob[pi];
  const int local = w - P.tile_begin;
  // bands of kTileBand tile rows walked column by column: the items of one
  // wave share a few L row panels and R column panels, so at large n the
  // panels a wave streams stay in L2 instead of every wave re-reading all of R
  constexpr int kTileBand = 8;
  const int rows = P.tile_count / P.tiles_n;  // tile rows of CM tiles
  const int band = local / (kTileBand * P.tiles_n);
  const int r0 = band * kTileBand;
  const int bh = rows - r0 < kTileBand ? rows - r0 : kTileBand;
  const int in = local - r0 * P.tiles_n;
  mt = (r0 + in % bh) * CM + rank;
  nt = in / bh;
}

__device__ __forceinline__ uint32_t pack_bf16x2(float a, float b) {
  __nv_bfloat162 v = __floats2bfloat162_rn(a, b);
  return *reinterpret_cast<uint32_t*>(&v);
}

// Epilogue of the 128 x BN accumulator tile at rows m0.., columns n0.., run by
// the epilogue warp of TMEM lane quarter q (rows m0 + 32q ... m0 + 32q + 31):
//
//   D = s * acc + beta * C + gamma * I
//
// written as f32 (D32) and as its bf16 split: hi = bf16(D), lo = bf16(D - hi)
// (Dhi, Dlo) and, with kLo2 (operands of split-bf16 x6 products),
// lo2 = bf16(D - hi - lo) (Dlo2).  `tmem` is
// the TMEM address of the quarter's first lane at the tile's first column;
// `wb` is this warp's 32 x kStride float transpose buffer.  Each 32-column
// chunk: tcgen05.ld gives lane l row (32q + l); the warp transposes it through
// shared memory so that every global access covers whole 128-byte row
// segments (8 lanes x 16 B per row, 4 rows per instruction) instead of one
// 16-byte piece of 32 different rows.  Returns this lane's sum of D^2 over its
// in-range elements.
template <int BN, int kStride, bool kLo2 = false>
__device__ __forceinline__ float epilogue_tile(const TcProblem& P, int m0, int n0, int q, int lane, float* wb,
                                               uint32_t tmem) {
  const int sub_r = lane >> 3;       // row within a group of 4
  const int sub_c = (lane & 7) * 4;  // first of this lane's 4 columns
  // the problem's fields in registers: the stores below could alias the
  // problem table as far as the compiler knows, which would force a reload
  // of every field after every store
  const float e_s = P.s, e_beta = P.beta, e_gamma = P.gamma;
  const int e_M = P.M, e_N = P.N;
  const int64_t e_ldc = P.ldc, e_ld32 = P.ldd32, e_ld16 = P.ldd16;
  const float* __restrict__ e_C = e_beta != 0.f ? P.C : nullptr;
  float* __restrict__ e_D32 = P.D32;
  bf16* __restrict__ e_Dhi = P.Dhi;
  bf16* __restrict__ e_Dlo = P.Dlo;
  bf16* __restrict__ e_Dlo2 = kLo2 && P.Dlo != nullptr ? P.Dlo2 : nullptr;
  float* __restrict__ e_Dt = P.Dt;
  float* __restrict__ e_DtT = P.DtT;
  const int64_t e_ldt = P.ldt;
  float frob = 0.f;
#pragma unroll 1
  for (int c0 = 0; c0 < BN; c0 += 32) {
    const int col0 = n0 + c0;
    if (col0 >= e_N) break;  // warp-uniform: no later chunk has columns either
    const int col = col0 + sub_c;
    const bool cols4 = col + 4 <= e_N;
    // the beta C term of all 8 row groups first, so that the loads overlap
    // one another and the TMEM load below
    float4 cv[8];
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      cv[g] = make_float4(0.f, 0.f, 0.f, 0.f);
      const int row = m0 + q * 32 + 4 * g + sub_r;
      if (e_C == nullptr || row >= e_M || col >= e_N) continue;
      const float* crow = e_C + static_cast<int64_t>(row) * e_ldc + col;
      if (cols4) {
        cv[g] = *reinterpret_cast<const float4*>(crow);
      } else {
        cv[g].x = crow[0];
        if (col + 1 < e_N) cv[g].y = crow[1];
        if (col + 2 < e_N) cv[g].z = crow[2];
      }
    }
    uint32_t r[32];
    tmem_ld_32x32b_x32(tmem + static_cast<uint32_t>(c0), r);
    tmem_wait_ld();
#pragma unroll
    for (int i = 0; i < 32; i += 4)
      *reinterpret_cast<float4*>(wb + lane * kStride + i) =
          make_float4(e_s * __uint_as_float(r[i]), e_s * __uint_as_float(r[i + 1]), e_s * __uint_as_float(r[i + 2]),
                      e_s * __uint_as_float(r[i + 3]));
    __syncwarp();
#pragma unroll
    for (int g = 0; g < 8; ++g) {
      const int rr = 4 * g + sub_r;
      const int row = m0 + q * 32 + rr;
      const float4 x4 = *reinterpret_cast<const float4*>(wb + rr * kStride + sub_c);
      if (row >= e_M || col >= e_N) continue;
      float v[4] = {x4.x, x4.y, x4.z, x4.w};
      if (e_C != nullptr) {
        v[0] += e_beta * cv[g].x;
        v[1] += e_beta * cv[g].y;
        v[2] += e_beta * cv[g].z;
        v[3] += e_beta * cv[g].w;
      }
      if (e_gamma != 0.f) {
#pragma unroll
        for (int t = 0; t < 4; ++t) v[t] += (row == col + t) ? e_gamma : 0.f;
      }
      if (e_Dt != nullptr || e_DtT != nullptr) {
        // TF32 forms of D for the next TF32 product (row form: whole 16-byte
        // pieces of a row; transposed form: 4 consecutive rows of one column)
        const float t0 = rna_tf32(v[0]), t1 = rna_tf32(v[1]), t2 = rna_tf32(v[2]), t3 = rna_tf32(v[3]);
        const float tv[4] = {t0, t1, t2, t3};
        if (e_Dt != nullptr) {
          if (cols4) {
            *reinterpret_cast<float4*>(e_Dt + static_cast<int64_t>(row) * e_ldt + col) = make_float4(t0, t1, t2, t3);
          } else {
#pragma unroll
            for (int t = 0; t < 4; ++t)
              if (col + t < e_N) e_Dt[static_cast<int64_t>(row) * e_ldt + col + t] = tv[t];
          }
        }
        if (e_DtT != nullptr) {
#pragma unroll
          for (int t = 0; t < 4; ++t)
            if (col + t < e_N) e_DtT[static_cast<int64_t>(col + t) * e_ldt + row] = tv[t];
        }
      }
      if (cols4) {
#pragma unroll
        for (int t = 0; t < 4; ++t) frob += v[t] * v[t];
        if (e_D32 != nullptr)
          *reinterpret_cast<float4*>(e_D32 + static_cast<int64_t>(row) * e_ld32 + col) =
              make_float4(v[0], v[1], v[2], v[3]);
        if (e_Dhi != nullptr) {
          const __nv_bfloat16 h0 = __float2bfloat16_rn(v[0]), h1 = __float2bfloat16_rn(v[1]);
          const __nv_bfloat16 h2 = __float2bfloat16_rn(v[2]), h3 = __float2bfloat16_rn(v[3]);
          __nv_bfloat162 ha, hb;
          ha.x = h0;
          ha.y = h1;
          hb.x = h2;
          hb.y = h3;
          const int64_t o16 = static_cast<int64_t>(row) * e_ld16 + col;
          *reinterpret_cast<uint2*>(e_Dhi + o16) =
              make_uint2(*reinterpret_cast<uint32_t*>(&ha), *reinterpret_cast<uint32_t*>(&hb));
          if (e_Dlo != nullptr)
            *reinterpret_cast<uint2*>(e_Dlo + o16) =
                make_uint2(pack_bf16x2(v[0] - __bfloat162float(h0), v[1] - __bfloat162float(h1)),
                           pack_bf16x2(v[2] - __bfloat162float(h2), v[3] - __bfloat162float(h3)));
          if (kLo2 && e_Dlo2 != nullptr) {
            const __nv_bfloat16 hh[4] = {h0, h1, h2, h3};
            float t[4];
#pragma unroll
            for (int u = 0; u < 4; ++u) {
              const float r = v[u] - __bfloat162float(hh[u]);
              t[u] = r - __bfloat162float(__float2bfloat16_rn(r));
            }
            *reinterpret_cast<uint2*>(e_Dlo2 + o16) = make_uint2(pack_bf16x2(t[0], t[1]), pack_bf16x2(t[2], t[3]));
          }
        }
      } else {
#pragma unroll
        for (int t = 0; t < 4; ++t) {
          if (col + t >= e_N) continue;
          frob += v[t] * v[t];
          if (e_D32 != nullptr) e_D32[static_cast<int64_t>(row) * e_ld32 + col + t] = v[t];
          if (e_Dhi != nullptr) {
            const int64_t o16 = static_cast<int64_t>(row) * e_ld16 + col + t;
            const __nv_bfloat16 h = __float2bfloat16_rn(v[t]);
            e_Dhi[o16] = h;
            if (e_Dlo != nullptr) e_Dlo[o16] = __float2bfloat16_rn(v[t] - __bfloat162float(h));
            if (kLo2 && e_Dlo2 != nullptr) {
              const float r = v[t] - __bfloat162float(h);
              e_Dlo2[o16] = __float2bfloat16_rn(r - __bfloat162float(__float2bfloat16_rn(r)));
            }
          }
        }
      }
    }
    __syncwarp();  // the buffer is rewritten by the next chunk
  }
  return frob;
}

}  // namespace tc
}  // namespace nsgb
