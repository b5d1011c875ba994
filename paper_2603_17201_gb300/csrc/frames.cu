// Host runtime of the projection search and loop fusion (Sec. IV-D): the
// frames object (resident keyframe features, Sec. IV-E) and the C ABI calls.
//
// pgo_frames_create copies the keyframes' features to the device once,
// bucketed per keyframe into a 64 x 48 grid over the image (a stable counting
// sort by cell, so features keep the caller's order within a cell), and keeps
// each keyframe's observed map point ids sorted for the fusion's skip test.
#include <cuda_runtime.h>

#include <algorithm>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <vector>

#include "internal.cuh"

using namespace pgo;

struct pgo_frames {
  int K = 0, F = 0;
  cudaStream_t stream = nullptr;
  char* arena = nullptr;
  FramesDev dev{};
  float min_x = 0, max_x = 0, min_y = 0, max_y = 0;
};

namespace {

pgo_status ffail(pgo_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof(buf), fmt, ap);
  va_end(ap);
  set_last_error(buf);
  return st;
}

template <class T>
bool fetch_arr(std::vector<T>& dst, const T* src, size_t n, int mem_space) {
  dst.resize(n);
  if (n == 0) return true;
  if (mem_space == PGO_MEM_DEVICE) return cudaMemcpy(dst.data(), src, n * sizeof(T), cudaMemcpyDeviceToHost) == cudaSuccess;
  std::memcpy(dst.data(), src, n * sizeof(T));
  return true;
}

size_t a256(size_t b) { return (b + 255) & ~size_t(255); }

bool al16(const void* p) { return (reinterpret_cast<uintptr_t>(p) & 15u) == 0; }

}  // namespace

extern "C" {

pgo_status pgo_frames_create(const pgo_frames_desc* d, pgo_frames** out) {
  if (!out) return ffail(PGO_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!d || !d->feat_ptr) return ffail(PGO_ERR_INVALID_ARG, "desc or feat_ptr is NULL");
  const int K = d->n_keyframes;
  if (K < 1 || K > 65535) return ffail(PGO_ERR_INVALID_ARG, "n_keyframes must be in [1, 65535] (got %d)", K);
  if (d->mem_space != PGO_MEM_HOST && d->mem_space != PGO_MEM_DEVICE)
    return ffail(PGO_ERR_INVALID_ARG, "mem_space must be PGO_MEM_HOST or PGO_MEM_DEVICE");
  if (!(d->max_x > d->min_x) || !(d->max_y > d->min_y) || !std::isfinite(d->max_x - d->min_x) ||
      !std::isfinite(d->max_y - d->min_y))
    return ffail(PGO_ERR_INVALID_ARG, "image bounds must satisfy min < max");
  std::vector<int> ptr(d->feat_ptr, d->feat_ptr + K + 1);
  if (ptr[0] != 0) return ffail(PGO_ERR_INVALID_ARG, "feat_ptr[0] must be 0");
  for (int k = 0; k < K; ++k)
    if (ptr[k + 1] < ptr[k]) return ffail(PGO_ERR_INVALID_ARG, "feat_ptr must be non-decreasing (keyframe %d)", k);
  const int F = ptr[K];
  if (F > 0 && (!d->uv || !d->octave || !d->desc)) return ffail(PGO_ERR_INVALID_ARG, "feature arrays are NULL");
  const int ms = d->mem_space;
  std::vector<float> uv;
  std::vector<int32_t> oct, mp;
  std::vector<uint32_t> desc;
  if (!fetch_arr(uv, d->uv, (size_t)F * 2, ms) || !fetch_arr(oct, d->octave, (size_t)F, ms) ||
      !fetch_arr(desc, d->desc, (size_t)F * 8, ms))
    return ffail(PGO_ERR_CUDA, "reading the feature arrays failed");
  if (d->map_point) {
    if (!fetch_arr(mp, d->map_point, (size_t)F, ms)) return ffail(PGO_ERR_CUDA, "reading map_point failed");
  } else {
    mp.assign((size_t)F, -1);
  }
  for (int f = 0; f < F; ++f)
    if (!std::isfinite(uv[2 * f]) || !std::isfinite(uv[2 * f + 1]))
      return ffail(PGO_ERR_INVALID_ARG, "feature %d: non-finite keypoint", f);
  const int cells = kGridCols * kGridRows;
  const double cw = ((double)d->max_x - d->min_x) / kGridCols, ch = ((double)d->max_y - d->min_y) / kGridRows;
  // stable counting sort of every keyframe's features by grid cell
  std::vector<int> cell_ptr((size_t)K * cells + 1, 0), cell_of((size_t)F);
  for (int k = 0; k < K; ++k)
    for (int f = ptr[k]; f < ptr[k + 1]; ++f) {
      int cx = (int)std::floor((uv[2 * f] - (double)d->min_x) / cw);
      int cy = (int)std::floor((uv[2 * f + 1] - (double)d->min_y) / ch);
      cx = std::min(std::max(cx, 0), kGridCols - 1);
      cy = std::min(std::max(cy, 0), kGridRows - 1);
      cell_of[f] = k * cells + cy * kGridCols + cx;
      cell_ptr[cell_of[f] + 1]++;
    }
  for (size_t c = 0; c < (size_t)K * cells; ++c) cell_ptr[c + 1] += cell_ptr[c];
  std::vector<int> fill(cell_ptr.begin(), cell_ptr.end() - 1);
  std::vector<float> s_uv((size_t)F * 2);
  std::vector<int> s_oct(F), s_orig(F);
  std::vector<uint32_t> s_desc((size_t)F * 8);
  for (int k = 0; k < K; ++k)
    for (int f = ptr[k]; f < ptr[k + 1]; ++f) {
      const int j = fill[cell_of[f]]++;
      s_uv[2 * j] = uv[2 * f];
      s_uv[2 * j + 1] = uv[2 * f + 1];
      s_oct[j] = oct[f];
      s_orig[j] = f - ptr[k];
      std::memcpy(&s_desc[(size_t)j * 8], &desc[(size_t)f * 8], 32);
    }
  // observed map point ids per keyframe, ascending
  std::vector<int> obs_ptr(K + 1, 0), obs;
  for (int k = 0; k < K; ++k) {
    const size_t b = obs.size();
    for (int f = ptr[k]; f < ptr[k + 1]; ++f)
      if (mp[f] >= 0) obs.push_back(mp[f]);
    std::sort(obs.begin() + b, obs.end());
    obs_ptr[k + 1] = (int)obs.size();
  }
  const size_t Fp = F > 0 ? F : 1, On = obs.empty() ? 1 : obs.size();
  size_t bytes = a256(sizeof(int) * (K + 1)) + a256(sizeof(int) * cell_ptr.size()) + a256(sizeof(float) * 2 * Fp) +
                 2 * a256(sizeof(int) * Fp) + a256(32 * Fp) + a256(sizeof(int) * Fp) + a256(sizeof(int) * (K + 1)) +
                 a256(sizeof(int) * On) + a256(sizeof(float) * 16 * K) + a256(sizeof(unsigned long long) * Fp);
  pgo_frames* Fr = new pgo_frames();
  Fr->K = K;
  Fr->F = F;
  Fr->stream = (cudaStream_t)d->stream;
  Fr->min_x = d->min_x;
  Fr->max_x = d->max_x;
  Fr->min_y = d->min_y;
  Fr->max_y = d->max_y;
  cudaError_t e = cudaMalloc(&Fr->arena, bytes);
  if (e != cudaSuccess) {
    cudaGetLastError();
    delete Fr;
    return ffail(e == cudaErrorMemoryAllocation ? PGO_ERR_OOM : PGO_ERR_CUDA, "cudaMalloc(%zu): %s", bytes,
                 cudaGetErrorString(e));
  }
  char* a = Fr->arena;
  auto take = [&](size_t n) {
    char* p = a;
    a += a256(n);
    return p;
  };
  FramesDev& D = Fr->dev;
  D.K = K;
  D.n_features = F;
  D.inv_cw = (float)(1.0 / cw);
  D.inv_ch = (float)(1.0 / ch);
  int* d_kf = reinterpret_cast<int*>(take(sizeof(int) * (K + 1)));
  int* d_cell = reinterpret_cast<int*>(take(sizeof(int) * cell_ptr.size()));
  float2* d_uv = reinterpret_cast<float2*>(take(sizeof(float) * 2 * Fp));
  int* d_oct = reinterpret_cast<int*>(take(sizeof(int) * Fp));
  int* d_orig = reinterpret_cast<int*>(take(sizeof(int) * Fp));
  uint4* d_desc = reinterpret_cast<uint4*>(take(32 * Fp));
  int* d_mp = reinterpret_cast<int*>(take(sizeof(int) * Fp));
  int* d_obs_ptr = reinterpret_cast<int*>(take(sizeof(int) * (K + 1)));
  int* d_obs = reinterpret_cast<int*>(take(sizeof(int) * On));
  D.kf_tab = reinterpret_cast<float*>(take(sizeof(float) * 16 * K));
  D.win = reinterpret_cast<unsigned long long*>(take(sizeof(unsigned long long) * Fp));
  D.kf_ptr = d_kf;
  D.cell_ptr = d_cell;
  D.uv = d_uv;
  D.oct = d_oct;
  D.orig = d_orig;
  D.desc = d_desc;
  D.mp = d_mp;
  D.obs_ptr = d_obs_ptr;
  D.obs_ids = d_obs;
  cudaStream_t s = Fr->stream;
  bool ok = true;
  auto up = [&](void* dst, const void* src, size_t n) {
    if (n) ok &= cudaMemcpyAsync(dst, src, n, cudaMemcpyHostToDevice, s) == cudaSuccess;
  };
  up(d_kf, ptr.data(), sizeof(int) * (K + 1));
  up(d_cell, cell_ptr.data(), sizeof(int) * cell_ptr.size());
  up(d_uv, s_uv.data(), sizeof(float) * 2 * F);
  up(d_oct, s_oct.data(), sizeof(int) * F);
  up(d_orig, s_orig.data(), sizeof(int) * F);
  up(d_desc, s_desc.data(), 32 * (size_t)F);
  up(d_mp, mp.data(), sizeof(int) * F);
  up(d_obs_ptr, obs_ptr.data(), sizeof(int) * (K + 1));
  up(d_obs, obs.data(), sizeof(int) * obs.size());
  ok &= cudaStreamSynchronize(s) == cudaSuccess;
  if (!ok) {
    cudaFree(Fr->arena);
    delete Fr;
    return ffail(PGO_ERR_CUDA, "uploading the frames failed");
  }
  *out = Fr;
  return PGO_OK;
}

void pgo_frames_destroy(pgo_frames* Fr) {
  if (!Fr) return;
  if (Fr->arena) {
    cudaStreamSynchronize(Fr->stream);
    cudaFree(Fr->arena);
  }
  delete Fr;
}

pgo_status pgo_project_match(pgo_frames* Fr, const pgo_match_params* prm, int32_t mode, const double* poses,
                             const uint8_t* matched, const pgo_points_desc* pts, int32_t* match, int32_t* dist,
                             int32_t* fuse) {
  if (!Fr || !prm || !pts) return ffail(PGO_ERR_INVALID_ARG, "frames, params or points is NULL");
  if (mode != PGO_MATCH_SEARCH && mode != PGO_MATCH_FUSE) return ffail(PGO_ERR_INVALID_ARG, "unknown mode %d", mode);
  if (!poses || !al16(poses)) return ffail(PGO_ERR_INVALID_ARG, "poses must be a non-NULL device array");
  const int P = pts->n_points;
  if (P < 0) return ffail(PGO_ERR_INVALID_ARG, "n_points must be >= 0");
  if (prm->n_levels < 1 || prm->n_levels > 32 || !(prm->scale_factor > 0.0f) || !(prm->th > 0.0f) ||
      prm->th_low < 0 || !std::isfinite(prm->scale_factor) || !std::isfinite(prm->th))
    return ffail(PGO_ERR_INVALID_ARG, "params: 1 <= n_levels <= 32, scale_factor > 0, th > 0, th_low >= 0");
  if (prm->min_x != Fr->min_x || prm->max_x != Fr->max_x || prm->min_y != Fr->min_y || prm->max_y != Fr->max_y)
    return ffail(PGO_ERR_INVALID_ARG, "params image bounds differ from the frames' grid bounds");
  if (P > 0) {
    if (!pts->xyz || !pts->desc || !pts->min_dist || !pts->max_dist || !pts->normal || !match || !dist)
      return ffail(PGO_ERR_INVALID_ARG, "NULL point or output array");
    if (!al16(pts->desc)) return ffail(PGO_ERR_INVALID_ARG, "point descriptors must be 16-byte aligned");
    if (mode == PGO_MATCH_FUSE && (!pts->id || !fuse))
      return ffail(PGO_ERR_INVALID_ARG, "fusion needs point ids and the fuse output");
    if ((long long)P * Fr->K > 0x7fffffffLL) return ffail(PGO_ERR_INVALID_ARG, "n_keyframes * n_points too large");
  }
  MatchParams mp;
  mp.fx = prm->fx; mp.fy = prm->fy; mp.cx = prm->cx; mp.cy = prm->cy;
  mp.min_x = prm->min_x; mp.max_x = prm->max_x; mp.min_y = prm->min_y; mp.max_y = prm->max_y;
  mp.scale_factor = prm->scale_factor; mp.th = prm->th; mp.cos_min = prm->cos_min;
  mp.n_levels = prm->n_levels; mp.th_low = prm->th_low;
  PointsDev pd;
  pd.n = P;
  pd.xyz = pts->xyz;
  pd.desc = pts->desc;
  pd.min_dist = pts->min_dist;
  pd.max_dist = pts->max_dist;
  pd.normal = pts->normal;
  pd.id = pts->id;
  const cudaError_t e = launch_project_match(Fr->dev, mp, mode, poses, mode == PGO_MATCH_SEARCH ? matched : nullptr,
                                             pd, match, dist, fuse, Fr->stream);
  if (e != cudaSuccess) return ffail(PGO_ERR_CUDA, "pgo_project_match: %s", cudaGetErrorString(e));
  return PGO_OK;
}

}  // extern "C"
