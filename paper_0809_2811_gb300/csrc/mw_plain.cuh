// mw_plain.cuh -- the plain GPU path: the straightforward CUDA mapping of the
// Sec. II.A sums that the batched, persistent and adjoint paths are measured
// against.  One thread per atom i walks i's neighbour row, keeps i's legs
// (r < a sig) in local memory, takes the pair term of each leg (half its
// energy and virial, the whole force on i; the partner does the same from
// its side) and the three-body term of every unordered leg pair (j, k) of
// centre i, scattering the forces on j and k with red.global and keeping the
// reaction on i.  Per-thread FP32 sums of E2, E3 and the virial go through
// the same per-box reduction as the other force kernels (FP64 across
// blocks).  No lane groups, no shared-memory leg table, no moment form: the
// per-centre work is the plain O(n^2) leg-pair loop.
#pragma once

#include "mw_device.cuh"

namespace mw {

constexpr int kPlainThreads = 128;

template <bool kCount>
__global__ void __launch_bounds__(kPlainThreads) k_force_plain(Dev d, FParams P) {
  if (block_stop(d)) return;
  const int par = (int)(d.g->step & 1ull);
  if (blockIdx.x == 0) {  // the rebuild (if any) is consumed
    for (int k = threadIdx.x; k < d.nbox; k += blockDim.x) d.bst[k].rebuild = 0;
    if (threadIdx.x == 0) {
      d.g->any_rebuild = 0;
      d.g->wpar = par;
    }
  }
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  float acc[8] = {0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f, 0.f};  // E2, E3, W xx yy zz xy xz yz
  int b = -1;
  if (i < d.N) {
    const uint4 qi = d.q[i];
    b = (int)qi.w;
    const Box& bx = d.box[b];
    const int cnt = min(d.nbr_cnt[i], d.W);
    float ux[kMaxLegsOverflow], uy[kMaxLegsOverflow], uz[kMaxLegsOverflow], tr[kMaxLegsOverflow],
        nde[kMaxLegsOverflow], ee[kMaxLegsOverflow], rr[kMaxLegsOverflow];
    float ax[kMaxLegsOverflow], ay[kMaxLegsOverflow], az[kMaxLegsOverflow];
    int jj[kMaxLegsOverflow];
    int nl = 0;
    float fx = 0.f, fy = 0.f, fz = 0.f;
    for (int s = 0; s < cnt; ++s) {
      const int j = d.nbr[(size_t)i * d.W + s];
      const uint4 qj = d.q[j];
      const float dx = fix_diff(qi.x, qj.x, bx.Lq[0]), dy = fix_diff(qi.y, qj.y, bx.Lq[1]),
                  dz = fix_diff(qi.z, qj.z, bx.Lq[2]);
      const float r2 = fmaf(dx, dx, fmaf(dy, dy, dz * dz));
      if (r2 >= P.rc2) continue;
      LegTerms lt;
      if (!leg_terms(r2, P, lt)) continue;
      if (nl >= kMaxLegsOverflow) {
        set_status(d.g, ST_LEGS);
        d.g->err_index = i;
        break;
      }
      ux[nl] = dx * lt.invr;
      uy[nl] = dy * lt.invr;
      uz[nl] = dz * lt.invr;
      tr[nl] = 2.0f * lt.invr;
      nde[nl] = lt.nde;
      ee[nl] = P.sle * lt.e3;
      rr[nl] = lt.r;
      jj[nl] = j;
      ax[nl] = ay[nl] = az[nl] = 0.f;
      // pair term: half energy, the whole force on i, half virial
      acc[0] = fmaf(0.5f, lt.phi, acc[0]);
      fx = fmaf(lt.dphi, ux[nl], fx);
      fy = fmaf(lt.dphi, uy[nl], fy);
      fz = fmaf(lt.dphi, uz[nl], fz);
      const float wv = -0.5f * lt.dphi * lt.r;
      acc[2] = fmaf(wv * ux[nl], ux[nl], acc[2]);
      acc[3] = fmaf(wv * uy[nl], uy[nl], acc[3]);
      acc[4] = fmaf(wv * uz[nl], uz[nl], acc[4]);
      acc[5] = fmaf(wv * ux[nl], uy[nl], acc[5]);
      acc[6] = fmaf(wv * ux[nl], uz[nl], acc[6]);
      acc[7] = fmaf(wv * uy[nl], uz[nl], acc[7]);
      ++nl;
    }
    if (kCount) {
      atomicAdd((unsigned long long*)&d.g->npairs, (unsigned long long)nl);
      atomicAdd((unsigned long long*)&d.g->ntrip, (unsigned long long)(nl * (nl - 1) / 2));
    }
    // three-body terms of centre i: every unordered leg pair once
    for (int j = 0; j < nl; ++j)
      for (int k = j + 1; k < nl; ++k) {
        const float c = fmaf(ux[j], ux[k], fmaf(uy[j], uy[k], uz[j] * uz[k]));
        const float D = c - P.c0;
        const float g = ee[j] * ee[k] * D;
        acc[1] = fmaf(g, D, acc[1]);
        const float aj = g * tr[j], bj = g * fmaf(c, tr[j], D * nde[j]);
        ax[j] = fmaf(-aj, ux[k], fmaf(bj, ux[j], ax[j]));
        ay[j] = fmaf(-aj, uy[k], fmaf(bj, uy[j], ay[j]));
        az[j] = fmaf(-aj, uz[k], fmaf(bj, uz[j], az[j]));
        const float ak = g * tr[k], bk = g * fmaf(c, tr[k], D * nde[k]);
        ax[k] = fmaf(-ak, ux[j], fmaf(bk, ux[k], ax[k]));
        ay[k] = fmaf(-ak, uy[j], fmaf(bk, uy[k], ay[k]));
        az[k] = fmaf(-ak, uz[j], fmaf(bk, uz[k], az[k]));
      }
    for (int k = 0; k < nl; ++k) {
      red_add_v4(d.f + jj[k], ax[k], ay[k], az[k]);
      fx -= ax[k];
      fy -= ay[k];
      fz -= az[k];
      const float rx = rr[k] * ux[k], ry = rr[k] * uy[k], rz = rr[k] * uz[k];
      acc[2] = fmaf(rx, ax[k], acc[2]);
      acc[3] = fmaf(ry, ay[k], acc[3]);
      acc[4] = fmaf(rz, az[k], acc[4]);
      acc[5] = fmaf(rx, ay[k], acc[5]);
      acc[6] = fmaf(rx, az[k], acc[6]);
      acc[7] = fmaf(ry, az[k], acc[7]);
    }
    red_add_v4(d.f + i, fx, fy, fz);
  }
  box_accumulate<8>(acc, b, [&](int bb) { return &d.bst[bb].ew[par][0]; });
}

}  // namespace mw
