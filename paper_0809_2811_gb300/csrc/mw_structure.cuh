// mw_structure.cuh -- structure analysis of the current positions (Sec. II.C):
// the pair histogram behind the radial distribution function g(r) and the
// angle histogram behind the angular distribution function (the angles at an
// atom between its n_c nearest neighbours).  Both read a neighbour list built
// at the current positions, so every pair within the list radius is in it.
// One thread per centre; counts of the block's first and last box are summed
// in shared memory (32-bit) and added to the per-box 64-bit histogram once per
// block, other boxes (small boxes only) go to global memory directly.
#pragma once

#include "mw_device.cuh"

namespace mw {

constexpr int kSThreads = 128;
constexpr int kAdfMax = 16;  // largest n_c of the angle histogram

struct BlockHist {
  unsigned* sh;  // [2][nbins]
  unsigned long long* glob;  // [nbox][nbins]
  int nbins, b_first, b_last;

  __device__ void begin(const Dev& d, unsigned* s, int nb, unsigned long long* g, int i0) {
    sh = s;
    glob = g;
    nbins = nb;
    b_first = (int)d.q[i0].w;
    b_last = (int)d.q[min(i0 + (int)blockDim.x, d.N) - 1].w;
    for (int k = threadIdx.x; k < 2 * nbins; k += blockDim.x) sh[k] = 0u;
    __syncthreads();
  }
  __device__ void add(int b, int k, unsigned c) {
    if (b == b_first) atomicAdd(sh + k, c);
    else if (b == b_last) atomicAdd(sh + nbins + k, c);
    else atomicAdd(glob + (size_t)b * nbins + k, (unsigned long long)c);
  }
  __device__ void end() {
    __syncthreads();
    for (int k = threadIdx.x; k < nbins; k += blockDim.x) {
      if (sh[k]) atomicAdd(glob + (size_t)b_first * nbins + k, (unsigned long long)sh[k]);
      if (b_last != b_first && sh[nbins + k]) atomicAdd(glob + (size_t)b_last * nbins + k, (unsigned long long)sh[nbins + k]);
    }
  }
};

// Pair histogram: every ordered pair (i, j), i != j, of one box with
// k dr <= r_ij < (k + 1) dr, k < nbins (nbins dr within the list radius).
__global__ void __launch_bounds__(kSThreads) k_pair_hist(Dev d, float inv_dr, float rmax2, int nbins,
                                                         unsigned long long* hist) {
  extern __shared__ unsigned s_hist[];
  const int i0 = (int)(blockIdx.x * blockDim.x);
  BlockHist h;
  h.begin(d, s_hist, nbins, hist, i0);
  const int i = i0 + (int)threadIdx.x;
  if (i < d.N) {
    const uint4 qi = d.q[i];
    const Box& bx = d.box[qi.w];
    const int cnt = min(d.nbr_cnt[i], d.W);
    const int* row = d.nbr + (size_t)i * d.W;
    for (int s = 0; s < cnt; ++s) {
      const uint4 qj = d.q[row[s]];
      const float dx = fix_diff(qi.x, qj.x, bx.Lq[0]), dy = fix_diff(qi.y, qj.y, bx.Lq[1]),
                  dz = fix_diff(qi.z, qj.z, bx.Lq[2]);
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (r2 < rmax2) {
        const int k = (int)(sqrtf(r2) * inv_dr);
        if (k < nbins) h.add((int)qi.w, k, 1u);
      }
    }
  }
  h.end();
}

// Angle histogram: for each atom k its nc nearest neighbours (from the list;
// fewer than nc within the list radius is counted in *short_rows), the angle
// theta_ikj at k for every ordered pair i != j of them, binned over
// [0, 180] degrees (180 itself in the last bin).
__global__ void __launch_bounds__(kSThreads) k_angle_hist(Dev d, int nc, int nbins, float inv_w,
                                                          unsigned long long* hist, int* short_rows) {
  extern __shared__ unsigned s_hist[];
  const int i0 = (int)(blockIdx.x * blockDim.x);
  BlockHist h;
  h.begin(d, s_hist, nbins, hist, i0);
  const int i = i0 + (int)threadIdx.x;
  if (i < d.N) {
    const uint4 qi = d.q[i];
    const Box& bx = d.box[qi.w];
    const int cnt = min(d.nbr_cnt[i], d.W);
    const int* row = d.nbr + (size_t)i * d.W;
    float br[kAdfMax];
    float ux[kAdfMax], uy[kAdfMax], uz[kAdfMax];
    int m = 0;
    for (int s = 0; s < cnt; ++s) {  // insertion into the nc nearest, ascending
      const uint4 qj = d.q[row[s]];
      const float dx = fix_diff(qi.x, qj.x, bx.Lq[0]), dy = fix_diff(qi.y, qj.y, bx.Lq[1]),
                  dz = fix_diff(qi.z, qj.z, bx.Lq[2]);
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (m == nc && !(r2 < br[nc - 1])) continue;
      int p = (m < nc) ? m++ : nc - 1;
      while (p > 0 && br[p - 1] > r2) {
        br[p] = br[p - 1];
        ux[p] = ux[p - 1];
        uy[p] = uy[p - 1];
        uz[p] = uz[p - 1];
        --p;
      }
      const float inv = rsqrtf(r2);
      br[p] = r2;
      ux[p] = dx * inv;
      uy[p] = dy * inv;
      uz[p] = dz * inv;
    }
    if (m < nc) {
      atomicAdd(short_rows, 1);
    } else {
      for (int a = 0; a < nc; ++a)
        for (int b = a + 1; b < nc; ++b) {
          float c = fmaf(ux[a], ux[b], fmaf(uy[a], uy[b], uz[a] * uz[b]));
          c = fminf(1.0f, fmaxf(-1.0f, c));
          const float th = acosf(c) * 57.29577951308232f;
          const int k = min(nbins - 1, (int)(th * inv_w));
          h.add((int)qi.w, k, 2u);  // the ordered pairs (a, b) and (b, a)
        }
    }
  }
  h.end();
}

}  // namespace mw
