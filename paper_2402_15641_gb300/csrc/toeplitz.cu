// Second stage of Algorithms 1 and 2 through the Toeplitz structure of A2.
//
// When the sensor rings sit at the slab centres (n_zs = mz over the volume
// height), the semicircle of ring h and radius l_m meets cell (slab k, radius
// bin l) exactly as the semicircle of ring h+1 meets cell (k+1, l):
//   A2[(h,m),(l,k)] = T[m, k - h, l].
// Forward:  p[n][h][m]  = sum_{l,d} T[m,d,l] Y1'[l][h+d][n]   (correlation in z)
// Adjoint:  F1[n][l][k] = sum_{m,d} T[m,d,l] P'[m][k-d][n]
// A CTA owns one block of TB output indices (m for the forward, l for the
// adjoint), one chunk of NC dense columns and every z position.  For each key
// (l, resp. m) it stages the input slab [z][NC] in shared memory, with zero
// halos so that shifted reads need no bounds checks, and applies the taps of
// that key: one tap = (offset d, band start o, W weights), i.e. W consecutive
// output indices fed from the same shifted slab read.  Accumulators live in
// registers; the warp-uniform band start selects a statically indexed update.
// No atomics: every output element is owned by one thread.
#include <algorithm>
#include <vector>

#include "common.cuh"
#include "devutil.cuh"

namespace {

constexpr int TB = SRT_TOEP_TB;
constexpr int NC = SRT_TOEP_NC;
constexpr int HG = 256 / NC;  // z positions per CTA pass (64)

__device__ __forceinline__ uint32_t smem_u32(const void* p) {
  return (uint32_t)__cvta_generic_to_shared(p);
}

template <typename V, int W>
__device__ __forceinline__ void load_taps(const V* __restrict__ w, int64_t e, float (&wv)[W]) {
  constexpr int WP = W;  // stored stride == W (4 or 8)
  const V* p = w + e * WP;
  if constexpr (sizeof(V) == 4) {
#pragma unroll
    for (int i = 0; i < W; i += 4) {
      const float4 t = __ldg(reinterpret_cast<const float4*>(p + i));
      wv[i] = t.x;
      wv[i + 1] = t.y;
      wv[i + 2] = t.z;
      wv[i + 3] = t.w;
    }
  } else {
#pragma unroll
    for (int i = 0; i < W; i += 4) {
      const uint2 t = __ldg(reinterpret_cast<const uint2*>(p + i));
      wv[i] = __uint_as_float(t.x << 16);
      wv[i + 1] = __uint_as_float(t.x & 0xffff0000u);
      wv[i + 2] = __uint_as_float(t.y << 16);
      wv[i + 3] = __uint_as_float(t.y & 0xffff0000u);
    }
  }
}

// acc[i][O + t] += w[t] * x[i] for the t with 0 <= O + t < TB.
template <int O, int W, int TH>
__device__ __forceinline__ void apply(float (&acc)[TH][TB], const float (&x)[TH],
                                      const float (&w)[W]) {
#pragma unroll
  for (int t = 0; t < W; ++t) {
    if (O + t >= 0 && O + t < TB) {  // compile-time: O, t are constants here
      constexpr int dummy = 0;
      (void)dummy;
#pragma unroll
      for (int i = 0; i < TH; ++i)
        acc[i][(O + t) & (TB - 1)] = fmaf(w[t], x[i], acc[i][(O + t) & (TB - 1)]);
    }
  }
}

template <int W, int TH>
__device__ __forceinline__ void apply_dyn(int o, float (&acc)[TH][TB], const float (&x)[TH],
                                          const float (&w)[W]) {
#define SRT_T_CASE(k)                                 \
  case k:                                             \
    if constexpr (k < TB + W - 1) apply<k - (W - 1), W, TH>(acc, x, w); \
    break;
  switch (o + (W - 1)) {
    SRT_T_CASE(0) SRT_T_CASE(1) SRT_T_CASE(2) SRT_T_CASE(3) SRT_T_CASE(4) SRT_T_CASE(5)
    SRT_T_CASE(6) SRT_T_CASE(7) SRT_T_CASE(8) SRT_T_CASE(9) SRT_T_CASE(10) SRT_T_CASE(11)
    SRT_T_CASE(12) SRT_T_CASE(13) SRT_T_CASE(14) SRT_T_CASE(15) SRT_T_CASE(16) SRT_T_CASE(17)
    SRT_T_CASE(18) SRT_T_CASE(19) SRT_T_CASE(20) SRT_T_CASE(21) SRT_T_CASE(22)
    default: break;
  }
#undef SRT_T_CASE
}

// x tiles: tile(key, c) = x + (key * nchunks + c) * npos * NC, rows [pos][NC].
template <typename V, int W, int TH>
__global__ void __launch_bounds__(256) k_toep(const int32_t* __restrict__ blk_seg,
                                              const int32_t* __restrict__ seg_key,
                                              const int32_t* __restrict__ seg_ent,
                                              const int32_t* __restrict__ meta,
                                              const V* __restrict__ w, const float* __restrict__ x,
                                              int npos, int halo, int rows, int nob, int ncols,
                                              int nchunks, float* __restrict__ out, int64_t sN,
                                              int64_t sP, int64_t sB) {
  extern __shared__ __align__(16) float slab_raw[];
  float4* slab = reinterpret_cast<float4*>(slab_raw);  // 2 buffers x rows x float4
  const int tid = threadIdx.x;
  const int nl = tid & (NC - 1), g = tid / NC;
  const int blk = blockIdx.x, c = blockIdx.y;
  // zero both buffers once: halos stay zero, the real rows are overwritten
  for (int r = tid; r < 2 * rows; r += 256) slab[r] = make_float4(0.f, 0.f, 0.f, 0.f);
  __syncthreads();
  float acc[TH][TB];
#pragma unroll
  for (int i = 0; i < TH; ++i)
#pragma unroll
    for (int t = 0; t < TB; ++t) acc[i][t] = 0.f;
  const int s0 = blk_seg[blk], s1 = blk_seg[blk + 1];
  auto issue = [&](int s, int buf) {
    const float4* src = reinterpret_cast<const float4*>(x) +
                        ((int64_t)seg_key[s] * nchunks + c) * npos;
    float4* dst = slab + buf * rows + halo;
    for (int r = tid; r < npos; r += 256)
      asm volatile("cp.async.cg.shared.global [%0], [%1], 16;\n" ::"r"(smem_u32(dst + r)),
                   "l"(src + r));
    asm volatile("cp.async.commit_group;\n" ::);
  };
  if (s0 < s1) issue(s0, 0);
  for (int s = s0; s < s1; ++s) {
    asm volatile("cp.async.wait_group 0;\n" ::);
    __syncthreads();  // slab s visible to all; slab s-1 no longer read
    if (s + 1 < s1) issue(s + 1, (s + 1 - s0) & 1);
    const float* S = reinterpret_cast<const float*>(slab + ((s - s0) & 1) * rows) + nl;
    const int e1 = seg_ent[s + 1];
    for (int e = seg_ent[s]; e < e1; ++e) {
      const int mt = __ldg(meta + e);
      const int d = (int)(int16_t)(mt & 0xffff), o = mt >> 16;
      float wv[W];
      load_taps<V, W>(w, e, wv);
      float xv[TH];
#pragma unroll
      for (int i = 0; i < TH; ++i) xv[i] = S[(halo + g + HG * i + d) * NC];
      apply_dyn<W, TH>(o, acc, xv, wv);
    }
  }
  const int n = c * NC + nl;
  if (n >= ncols) return;
#pragma unroll
  for (int i = 0; i < TH; ++i) {
    const int pos = g + HG * i;
    if (pos >= npos) continue;
#pragma unroll
    for (int t = 0; t < TB; ++t) {
      const int ob = blk * TB + t;
      if (ob < nob) out[n * sN + pos * sP + ob * sB] = acc[i][t];
    }
  }
}

// tiles from rows: out[key][c][pos][NC] = in[n][key][pos], n = c*NC + lane.
__global__ void __launch_bounds__(256) k_tiles_rows(const float* __restrict__ in, int nkey,
                                                    int npos, int ncols,
                                                    float4* __restrict__ out) {
  const int key = blockIdx.x, c = blockIdx.y;
  const int nchunks = gridDim.y;
  for (int pos = threadIdx.x; pos < npos; pos += blockDim.x) {
    float v[NC];
#pragma unroll
    for (int j = 0; j < NC; ++j) {
      const int n = c * NC + j;
      v[j] = n < ncols ? __ldg(in + ((int64_t)n * nkey + key) * npos + pos) : 0.f;
    }
    out[((int64_t)key * nchunks + c) * npos + pos] = make_float4(v[0], v[1], v[2], v[3]);
  }
}

// tiles from columns: out[key][c][pos][NC] = in[n][pos][key]; one block per
// (chunk, 8 positions, 128 keys), transposed through shared memory.
__global__ void __launch_bounds__(256) k_tiles_cols(const float* __restrict__ in, int nkey,
                                                    int npos, int ncols, int nchunks,
                                                    float4* __restrict__ out) {
  constexpr int PP = 8, KK = 128;
  __shared__ float t[NC][PP][KK + 1];
  const int c = blockIdx.x, p0 = blockIdx.y * PP, k0 = blockIdx.z * KK;
  for (int i = threadIdx.x; i < NC * PP * KK; i += 256) {
    const int kk = i % KK, pp = (i / KK) % PP, j = i / (KK * PP);
    const int n = c * NC + j, pos = p0 + pp, key = k0 + kk;
    t[j][pp][kk] = (n < ncols && pos < npos && key < nkey)
                       ? __ldg(in + ((int64_t)n * npos + pos) * nkey + key)
                       : 0.f;
  }
  __syncthreads();
  for (int i = threadIdx.x; i < PP * KK; i += 256) {
    const int pp = i % PP, kk = i / PP;
    const int pos = p0 + pp, key = k0 + kk;
    if (pos < npos && key < nkey)
      out[((int64_t)key * nchunks + c) * npos + pos] =
          make_float4(t[0][pp][kk], t[1][pp][kk], t[2][pp][kk], t[3][pp][kk]);
  }
}

template <typename V, int W, int TH>
int launch_toep(const SrtTapList& L, const V* w, int npos, int halo, int nob, int ncols,
                const float* x, float* out, int64_t sN, int64_t sP, int64_t sB, cudaStream_t st) {
  const int nchunks = (ncols + NC - 1) / NC;
  const int rows = 2 * halo + (npos > HG * TH ? npos : HG * TH);
  const int smem = 2 * rows * 16;
  if (smem > 227 * 1024) return SRT_ERR_GEOMETRY;
  static int attr = 0;
  if (smem > 48 * 1024 && attr < smem) {
    SRT_CUDA_TRY(cudaFuncSetAttribute(k_toep<V, W, TH>,
                                      cudaFuncAttributeMaxDynamicSharedMemorySize, smem));
    attr = smem;
  }
  dim3 grid(L.nblk, nchunks);
  k_toep<V, W, TH><<<grid, 256, smem, st>>>(L.blk_seg, L.seg_key, L.seg_ent, L.meta, w, x, npos,
                                             halo, rows, nob, ncols, nchunks, out, sN, sP, sB);
  SRT_CUDA_TRY(cudaGetLastError());
  return SRT_OK;
}

template <typename V, int W>
int pick_th(const SrtTapList& L, const V* w, int npos, int halo, int nob, int ncols,
            const float* x, float* out, int64_t sN, int64_t sP, int64_t sB, cudaStream_t st) {
  if (npos <= HG) return launch_toep<V, W, 1>(L, w, npos, halo, nob, ncols, x, out, sN, sP, sB, st);
  if (npos <= 2 * HG) return launch_toep<V, W, 2>(L, w, npos, halo, nob, ncols, x, out, sN, sP, sB, st);
  if (npos <= 4 * HG) return launch_toep<V, W, 4>(L, w, npos, halo, nob, ncols, x, out, sN, sP, sB, st);
  if (npos <= 8 * HG) return launch_toep<V, W, 8>(L, w, npos, halo, nob, ncols, x, out, sN, sP, sB, st);
  return SRT_ERR_GEOMETRY;
}

// ---------------------------------------------------------------- host build
struct Piece {
  int key, d, o;     // key (slab), offset, band start within the block
  int blk;           // output block
  int src;           // index of the first weight in the host weight array
  int len;           // weights in the band piece
};

template <typename V>
int upload(const std::vector<Piece>& pcs, const std::vector<V>& wsrc, int nblk, int W,
           SrtTapList* L, V** wout, int64_t* bytes) {
  // pieces are sorted by (blk, key, d)
  std::vector<int32_t> blk_seg(nblk + 1, 0), seg_key, seg_ent, meta;
  std::vector<V> wv;
  meta.reserve(pcs.size());
  wv.reserve(pcs.size() * W);
  size_t i = 0;
  for (int b = 0; b < nblk; ++b) {
    blk_seg[b] = (int32_t)seg_key.size();
    while (i < pcs.size() && pcs[i].blk == b) {
      const int key = pcs[i].key;
      seg_key.push_back(key);
      seg_ent.push_back((int32_t)meta.size());
      while (i < pcs.size() && pcs[i].blk == b && pcs[i].key == key) {
        const Piece& p = pcs[i];
        meta.push_back((int32_t)((uint32_t)(uint16_t)(int16_t)p.d | ((uint32_t)p.o << 16)));
        for (int t = 0; t < W; ++t) wv.push_back(t < p.len ? wsrc[p.src + t] : V(0));
        ++i;
      }
    }
  }
  blk_seg[nblk] = (int32_t)seg_key.size();
  seg_ent.push_back((int32_t)meta.size());
  L->nblk = nblk;
  L->W = L->WP = W;
  L->nseg = (int64_t)seg_key.size();
  L->nent = (int64_t)meta.size();
  SRT_TRY(srt_dmalloc(&L->blk_seg, nblk + 1, bytes));
  SRT_TRY(srt_dmalloc(&L->seg_key, L->nseg, bytes));
  SRT_TRY(srt_dmalloc(&L->seg_ent, L->nseg + 1, bytes));
  SRT_TRY(srt_dmalloc(&L->meta, L->nent, bytes));
  SRT_TRY(srt_dmalloc(wout, L->nent * W, bytes));
  SRT_CUDA_TRY(cudaMemcpy(L->blk_seg, blk_seg.data(), 4 * blk_seg.size(), cudaMemcpyHostToDevice));
  if (!seg_key.empty())
    SRT_CUDA_TRY(cudaMemcpy(L->seg_key, seg_key.data(), 4 * seg_key.size(), cudaMemcpyHostToDevice));
  SRT_CUDA_TRY(cudaMemcpy(L->seg_ent, seg_ent.data(), 4 * seg_ent.size(), cudaMemcpyHostToDevice));
  if (!meta.empty()) {
    SRT_CUDA_TRY(cudaMemcpy(L->meta, meta.data(), 4 * meta.size(), cudaMemcpyHostToDevice));
    SRT_CUDA_TRY(cudaMemcpy(*wout, wv.data(), sizeof(V) * wv.size(), cudaMemcpyHostToDevice));
  }
  return SRT_OK;
}

// Split a run of consecutive output indices [a, a+len) (weights at src) into
// pieces of at most W and attach each piece to every block it meets.
void add_run(std::vector<Piece>& out, int key, int d, int a, int len, int src, int W, int nob) {
  for (int p = 0; p < len; p += W) {
    const int s = a + p, n = std::min(W, len - p);
    const int b0 = s / TB, b1 = (s + n - 1) / TB;
    for (int b = b0; b <= b1 && b * TB < nob; ++b)
      out.push_back(Piece{key, d, s - b * TB, b, src + p, n});
  }
}

template <typename V>
int build_lists(srt_plan_s* plan, const std::vector<int32_t>& rp, const std::vector<int32_t>& cl,
                const std::vector<V>& val, int64_t* bytes) {
  const srt_geometry& g = plan->g;
  const int nl = g.n_ell, mz = g.mz, mz2 = 2 * mz - 1;
  const int nblk = (nl + TB - 1) / TB;
  // forward: for every cell (l, d) the run of shells m crossing it
  const int ncell = nl * mz2;
  std::vector<int32_t> cnt(ncell + 1, 0);
  for (size_t e = 0; e < cl.size(); ++e) cnt[cl[e] + 1]++;
  for (int c = 0; c < ncell; ++c) cnt[c + 1] += cnt[c];
  std::vector<int32_t> cm(cl.size());
  std::vector<V> cv(cl.size());
  {
    std::vector<int32_t> cur(cnt.begin(), cnt.end() - 1);
    for (int m = 0; m < nl; ++m)
      for (int e = rp[m]; e < rp[m + 1]; ++e) {
        const int at = cur[cl[e]]++;
        cm[at] = m;
        cv[at] = val[e];
      }
  }
  int maxrun = 1;
  for (int c = 0; c < ncell; ++c) {
    int run = 0;
    for (int e = cnt[c]; e < cnt[c + 1]; ++e) {
      run = (e > cnt[c] && cm[e] == cm[e - 1] + 1) ? run + 1 : 1;
      maxrun = std::max(maxrun, run);
    }
  }
  const int WF = maxrun <= 4 ? 4 : 8;
  std::vector<Piece> fw;
  for (int c = 0; c < ncell; ++c) {
    const int l = c / mz2, d = c % mz2 - (mz - 1);
    int e = cnt[c];
    while (e < cnt[c + 1]) {
      int f = e + 1;
      while (f < cnt[c + 1] && cm[f] == cm[f - 1] + 1) ++f;
      add_run(fw, l, d, cm[e], f - e, e, WF, nl);
      e = f;
    }
  }
  std::sort(fw.begin(), fw.end(), [](const Piece& a, const Piece& b) {
    if (a.blk != b.blk) return a.blk < b.blk;
    if (a.key != b.key) return a.key < b.key;
    return a.d < b.d;
  });
  V* wf = nullptr;
  SRT_TRY(upload<V>(fw, cv, nblk, WF, &plan->tf, &wf, bytes));
  if (sizeof(V) == 4) plan->tf.w32 = reinterpret_cast<float*>(wf);
  else plan->tf.w16 = reinterpret_cast<uint16_t*>(wf);

  // adjoint: for every (m, d) the run of radius bins l crossing it.  Row m of
  // T lists (l, d) by l, then d; regroup by d.
  std::vector<Piece> aw;
  std::vector<V> av;
  std::vector<int32_t> ord;
  for (int m = 0; m < nl; ++m) {
    ord.clear();
    for (int e = rp[m]; e < rp[m + 1]; ++e) ord.push_back(e);
    std::stable_sort(ord.begin(), ord.end(), [&](int a, int b) {
      return cl[a] % mz2 < cl[b] % mz2;  // by d, then l (stable)
    });
    size_t i = 0;
    while (i < ord.size()) {
      const int d = cl[ord[i]] % mz2 - (mz - 1);
      size_t j = i + 1;
      while (j < ord.size() && cl[ord[j]] % mz2 == cl[ord[i]] % mz2 &&
             cl[ord[j]] / mz2 == cl[ord[j - 1]] / mz2 + 1)
        ++j;
      const int src = (int)av.size();
      for (size_t k = i; k < j; ++k) av.push_back(val[ord[k]]);
      add_run(aw, m, -d, cl[ord[i]] / mz2, (int)(j - i), src, 4, nl);  // reads row k - d
      i = j;
    }
  }
  std::sort(aw.begin(), aw.end(), [](const Piece& a, const Piece& b) {
    if (a.blk != b.blk) return a.blk < b.blk;
    if (a.key != b.key) return a.key < b.key;
    return a.d < b.d;
  });
  V* wa = nullptr;
  SRT_TRY(upload<V>(aw, av, nblk, 4, &plan->ta, &wa, bytes));
  if (sizeof(V) == 4) plan->ta.w32 = reinterpret_cast<float*>(wa);
  else plan->ta.w16 = reinterpret_cast<uint16_t*>(wa);
  return SRT_OK;
}

}  // namespace

void srt_taps_free(SrtTapList* t) {
  cudaFree(t->blk_seg);
  cudaFree(t->seg_key);
  cudaFree(t->seg_ent);
  cudaFree(t->meta);
  cudaFree(t->w32);
  cudaFree(t->w16);
  *t = SrtTapList();
}

int srt_build_toeplitz(srt_plan_s* plan, const SrtCsr& T, int64_t* bytes) {
  std::vector<int32_t> rp(T.rows + 1), cl(T.nnz);
  SRT_CUDA_TRY(cudaMemcpy(rp.data(), T.rowptr, 4 * rp.size(), cudaMemcpyDeviceToHost));
  if (T.nnz) SRT_CUDA_TRY(cudaMemcpy(cl.data(), T.col, 4 * cl.size(), cudaMemcpyDeviceToHost));
  if (plan->g.weight_dtype == SRT_BF16) {
    std::vector<uint16_t> v(T.nnz);
    if (T.nnz) SRT_CUDA_TRY(cudaMemcpy(v.data(), T.v16, 2 * v.size(), cudaMemcpyDeviceToHost));
    return build_lists<uint16_t>(plan, rp, cl, v, bytes);
  }
  std::vector<float> v(T.nnz);
  if (T.nnz) SRT_CUDA_TRY(cudaMemcpy(v.data(), T.v32, 4 * v.size(), cudaMemcpyDeviceToHost));
  return build_lists<float>(plan, rp, cl, v, bytes);
}

int srt_toep_apply(const SrtTapList& L, int wdt, int npos, int halo, int nob, int ncols,
                   const float* x, float* out, int64_t sN, int64_t sP, int64_t sB,
                   cudaStream_t st) {
  if (wdt == SRT_BF16) {
    if (L.W == 4) return pick_th<uint16_t, 4>(L, L.w16, npos, halo, nob, ncols, x, out, sN, sP, sB, st);
    return pick_th<uint16_t, 8>(L, L.w16, npos, halo, nob, ncols, x, out, sN, sP, sB, st);
  }
  if (L.W == 4) return pick_th<float, 4>(L, L.w32, npos, halo, nob, ncols, x, out, sN, sP, sB, st);
  return pick_th<float, 8>(L, L.w32, npos, halo, nob, ncols, x, out, sN, sP, sB, st);
}

int srt_tiles_from_rows(const float* in, int nkey, int npos, int ncols, float* out,
                        cudaStream_t st) {
  const int nchunks = (ncols + NC - 1) / NC;
  if (nchunks > 65535) return SRT_ERR_ARG;
  dim3 grid(nkey, nchunks);
  k_tiles_rows<<<grid, 256, 0, st>>>(in, nkey, npos, ncols, reinterpret_cast<float4*>(out));
  SRT_CUDA_TRY(cudaGetLastError());
  return SRT_OK;
}

int srt_tiles_from_cols(const float* in, int nkey, int npos, int ncols, float* out,
                        cudaStream_t st) {
  const int nchunks = (ncols + NC - 1) / NC;
  dim3 grid(nchunks, (npos + 7) / 8, (nkey + 127) / 128);
  if (grid.y > 65535 || grid.z > 65535) return SRT_ERR_ARG;
  k_tiles_cols<<<grid, 256, 0, st>>>(in, nkey, npos, ncols, nchunks,
                                     reinterpret_cast<float4*>(out));
  SRT_CUDA_TRY(cudaGetLastError());
  return SRT_OK;
}
