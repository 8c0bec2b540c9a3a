// mw_api.cu -- the C ABI of libmw (declared in include/mw.h).
//
// Host side: validates arguments, owns device buffers, sequences the kernels
// of mw_device.cuh on the system's stream, captures one MD step into a CUDA
// graph (graph engine) or launches the persistent cooperative kernel
// (persistent engine), and recovers from neighbour-list overflow.
#include <cuda_runtime.h>

#include <algorithm>
#include <atomic>
#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstdlib>
#include <cstring>
#include <string>
#include <vector>

#include <nvtx3/nvToolsExt.h>

#include "mw.h"
#include "mw_device.cuh"
#include "mw_persistent.cuh"
#include "mw_adjoint.cuh"
#include "mw_structure.cuh"
#include "mw_species.cuh"
#include "mw_plain.cuh"

static_assert(MW_MAX_SPECIES == mw::kMaxSpecies, "species limit of the header and the kernels");

using namespace mw;

namespace {

thread_local std::string g_err;

mw_status fail(mw_status st, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  g_err = buf;
  return st;
}

#define MW_CUDA(call)                                                                              \
  do {                                                                                             \
    cudaError_t e_ = (call);                                                                       \
    if (e_ != cudaSuccess) return fail(MW_ECUDA, "%s failed: %s", #call, cudaGetErrorString(e_)); \
  } while (0)

int div_up(long long a, int b) { return (int)((a + b - 1) / b); }

constexpr int kThreads = 128;

}  // namespace

struct mw_system {
  int nbox = 0, N = 0, W = 0, ncell = 0, ncell_cap = 0;
  std::vector<int> n, off;
  std::vector<Box> boxes;
  mw_params prm{};
  double mass = 18.015, skin = 1.0;
  cudaStream_t stream = nullptr;
  cudaStream_t cap_stream = nullptr;  // second stream for capturing conditional bodies
  // mw_set_state's velocity copy runs on copy_stream beside the force call at
  // the new positions; copy_ev[1] marks it done, and v_pending says that the
  // velocities in stage2 are still to be loaded (before the thermo snapshot)
  cudaStream_t copy_stream = nullptr;
  cudaEvent_t copy_ev[2] = {nullptr, nullptr};
  bool v_pending = false;
  bool own_stream = false;
  bool list_built = false;
  // the atom order and neighbour lists are current for the geometry and
  // parameters (set by a completed force call; cleared by anything that
  // flags every box for a rebuild, by a failed run, by isobaric steps):
  // mw_set_state may then keep them (k_load_state_keep)
  bool order_ok = false;
  double* eout = nullptr;  // 9 * nbox doubles: energies + virials staging
  Dev d{};
  FParams fp{};
  Integ integ{};
  bool integ_set = false;
  int* boxid = nullptr;  // user-order box id per atom
  AdjDev adj{};  // adjoint buffers (dL/dF, dL/dx accumulators, per-box sums)
  // state
  bool state_set = false;
  bool forces_valid = false;
  bool need_prime = true;  // thermostat start half must be recomputed before the next step
  bool record_pending = false;  // steps ran since the last thermo record was written
  bool boxes_stale = false;     // an isobaric run changed the device's box geometry since the last pull
  // several species (nsp > 1): the caller's table and the largest pair cutoff
  int nsp = 1;
  bool sp_moment = false;  // the table factors into leg weights: moment kernel (k_force_sp)
  std::vector<mw_params> sp_table;
  double sp_rc_max = 0;
  int *typ_buf = nullptr, *ttyp_buf = nullptr, *utyp_buf = nullptr;
  SpPair* sp_pair_buf = nullptr;
  float2* sp_tri_buf = nullptr;
  long long regrids = 0;        // cell grids laid out again because an isobaric box left its grid
  unsigned long long* ana = nullptr;  // structure-analysis histograms (grow-only)
  size_t ana_cap = 0;
  long long host_step = 0;
  int engine = MW_ENGINE_AUTO, engine_used = MW_ENGINE_GRAPH;
  int tuned_engine = -1;
  int force_shape = 0;  // launch shape of k_force (force_shape_lanes / force_shape_blocks)
  int count_terms = 0;
  long long npairs = 0, ntrip = 0;
  // graph engine
  cudaGraphExec_t graph1 = nullptr, graphK = nullptr;
  int graphK_steps = 0;
  bool graph_dirty = true;
  // persistent engine
  int pers_blocks = 0;
  int pers_blocks_limit = 0;  // 0 = as many as can be co-resident
  unsigned long long wait_ns = kBarrierTimeoutNs;  // limit of each device-side wait
  std::vector<int> cell_box_host;
  std::vector<void*> allocs;
  // pinned host staging for the small device-to-host reads (the Global
  // status block, then nbox thermo records), so that they need no staging copy
  void* hpin = nullptr;
  Global* gpin() { return static_cast<Global*>(hpin); }
  double* thpin() { return reinterpret_cast<double*>(static_cast<char*>(hpin) + kPinThermoOff); }
  static constexpr size_t kPinThermoOff = (sizeof(Global) + 63) / 64 * 64;
  // the status block as ensure_forces last read it, when nothing has run since
  bool g_known_valid = false;
  Global g_known{};
};

namespace {

// Host-side NVTX range over one public call (named in profiler timelines;
// inert without a profiler attached).
struct Range {
  explicit Range(const char* name) { nvtxRangePushA(name); }
  ~Range() { nvtxRangePop(); }
};

// defined in mw_persistent_host.inc / mw_adjoint_host.inc
mw_status persistent_func_attrs();
bool persistent_available(mw_system* s);
mw_status run_persistent_engine(mw_system* s, int nsteps, mw_thermo* last, bool* fetched);
mw_status enqueue_persistent(mw_system* s, int nsteps);
mw_status adjoint_alloc(mw_system* s);
mw_status prime_thermostat(mw_system* s);

template <class T>
mw_status dalloc(mw_system* s, T** p, size_t count) {
  void* q = nullptr;
  if (count == 0) count = 1;
  cudaError_t e = cudaMalloc(&q, count * sizeof(T));
  if (e != cudaSuccess) return fail(MW_ENOMEM, "cudaMalloc of %zu bytes failed: %s", count * sizeof(T), cudaGetErrorString(e));
  s->allocs.push_back(q);
  *p = (T*)q;
  return MW_OK;
}

void dfree(mw_system* s, void* p) {
  if (!p) return;
  auto it = std::find(s->allocs.begin(), s->allocs.end(), p);
  if (it != s->allocs.end()) s->allocs.erase(it);
  cudaFree(p);
}

// Largest interaction range: a sigma, or the widest pair's under several species.
double cutoff(const mw_system* s) { return s->nsp > 1 ? s->sp_rc_max : s->prm.a * s->prm.sigma; }
double r_list(const mw_system* s) { return cutoff(s) + s->skin; }

mw_status check_params(const mw_params* p) {
  if (!p) return fail(MW_EINVAL, "params is NULL");
  const double v[] = {p->lambda, p->epsilon, p->sigma, p->a, p->gamma, p->A, p->B, p->cos_theta0};
  for (double x : v)
    if (!std::isfinite(x)) return fail(MW_EINVAL, "non-finite parameter");
  if (p->sigma <= 0 || p->a <= 0 || p->epsilon < 0 || p->lambda < 0 || p->gamma < 0)
    return fail(MW_EINVAL, "parameters out of range (sigma, a > 0; epsilon, lambda, gamma >= 0)");
  if (p->p < 0 || p->p > 16 || p->q < 0 || p->q > 16) return fail(MW_EINVAL, "p and q must be in [0, 16]");
  return MW_OK;
}

void make_fparams(mw_system* s) {
  const mw_params& p = s->prm;
  const double rc = cutoff(s), rl = r_list(s);  // the widest pair under several species
  const double l2e = 1.4426950408889634;
  FParams& f = s->fp;
  f.rc = (float)rc;
  f.rc2 = (float)(rc * rc);
  f.rl2 = (float)(rl * rl);
  f.sig = (float)p.sigma;
  f.sig_l2e = (float)(p.sigma * l2e);
  f.gsig_l2e = (float)(p.gamma * p.sigma * l2e);
  f.gsig = (float)(p.gamma * p.sigma);
  f.Aeps = (float)(p.A * p.epsilon);
  f.B = (float)p.B;
  f.c0 = (float)p.cos_theta0;
  f.sle = (float)std::sqrt(p.lambda * p.epsilon);
  f.p = p.p;
  f.q = p.q;
  f.rc_lo = (float)(rc - (double)f.rc);
  f.sig_lo = (float)(p.sigma - (double)f.sig);
  f.sig_l2e_lo = (float)(p.sigma * l2e - (double)f.sig_l2e);
  f.gsig_l2e_lo = (float)(p.gamma * p.sigma * l2e - (double)f.gsig_l2e);
  f.B_lo = (float)(p.B - (double)f.B);
}

// The device's box geometry (scaled every step by the barostat of an
// isobaric run) back into the host copy, before host code reads or uploads it.
mw_status pull_boxes(mw_system* s) {
  if (!s->boxes_stale) return MW_OK;
  MW_CUDA(cudaMemcpyAsync(s->boxes.data(), s->d.box, sizeof(Box) * s->nbox, cudaMemcpyDeviceToHost, s->stream));
  MW_CUDA(cudaStreamSynchronize(s->stream));
  s->boxes_stale = false;
  return MW_OK;
}

// Cell grids of all boxes for the current list radius; returns the total.
// Under an isobaric integrator the cells get kCellMargin r_list of width at
// the smaller of the current and the coming edges, so that a box may shrink
// by about a tenth before its grid has to be laid out again.
mw_status layout_cells(mw_system* s, int* ncell_out) {
  mw_status st;
  if ((st = pull_boxes(s)) != MW_OK) return st;
  const double rl = r_list(s);
  const bool npt = s->integ.kind == TH_NPT;
  const double cw = npt ? kCellMargin * rl : rl;
  long long total = 0;
  for (int b = 0; b < s->nbox; ++b) {
    Box& bx = s->boxes[b];
    for (int k = 0; k < 3; ++k) {
      const double L = (npt && bx.Ln[k] > 0) ? std::min(bx.L[k], bx.Ln[k]) : bx.L[k];
      if (L < 2.0 * rl)
        return fail(MW_EBOX, "box %d edge %d = %g A is shorter than 2 r_list = %g A", b, k, L, 2 * rl);
      bx.nc[k] = std::max(1, (int)std::floor(L / cw));
    }
    bx.cell_off = (int)total;
    total += (long long)bx.nc[0] * bx.nc[1] * bx.nc[2];
  }
  if (total > (1ll << 30)) return fail(MW_EINVAL, "too many cells");
  *ncell_out = (int)total;
  return MW_OK;
}

// Neighbour row widths are whole 128-byte lines (32 entries): rows that
// straddle lines cost the force kernel ~50 % more DRAM reads for the same
// entries (ncu at 2^20 atoms: 184 MB per launch at 64, 96 or 128 slots,
// 246-276 MB at 56, 72 or 80).
int row_width(int w) { return std::max(32, (w + 31) / 32 * 32); }

int initial_width(const mw_system* s) {
  double rho = 0;
  for (int b = 0; b < s->nbox; ++b) {
    const Box& bx = s->boxes[b];
    rho = std::max(rho, bx.n / (bx.L[0] * bx.L[1] * bx.L[2]));
  }
  const double rl = r_list(s);
  const double expect = rho * 4.18879020478639 * rl * rl * rl;
  int w = (int)std::ceil(1.5 * expect + 16);
  return std::min(row_width(w), 1024);
}

mw_status upload_boxes(mw_system* s) {
  MW_CUDA(cudaMemcpyAsync((void*)s->d.box, s->boxes.data(), sizeof(Box) * s->nbox, cudaMemcpyHostToDevice, s->stream));
  return MW_OK;
}

mw_status upload_integ(mw_system* s) {
  MW_CUDA(cudaMemcpyAsync((void*)s->d.integ, &s->integ, sizeof(Integ), cudaMemcpyHostToDevice, s->stream));
  return MW_OK;
}

mw_status alloc_cells(mw_system* s) {
  mw_status st;
  if (s->ncell > s->ncell_cap) {  // grow only; a smaller grid reuses the arrays
    dfree(s, s->d.cell_cnt);
    dfree(s, s->d.cell_start);
    dfree(s, s->d.cell_box);
    s->d.cell_cnt = s->d.cell_start = s->d.cell_box = nullptr;
    if ((st = dalloc(s, &s->d.cell_cnt, s->ncell)) != MW_OK) return st;
    if ((st = dalloc(s, &s->d.cell_start, s->ncell + 1)) != MW_OK) return st;
    if ((st = dalloc(s, &s->d.cell_box, s->ncell)) != MW_OK) return st;
    s->ncell_cap = s->ncell;
  }
  MW_CUDA(cudaMemsetAsync(s->d.cell_cnt, 0, sizeof(int) * s->ncell, s->stream));
  s->cell_box_host.resize(s->ncell);
  for (int b = 0; b < s->nbox; ++b) {
    const Box& bx = s->boxes[b];
    const int nc = bx.nc[0] * bx.nc[1] * bx.nc[2];
    for (int k = 0; k < nc; ++k) s->cell_box_host[bx.cell_off + k] = b;
  }
  MW_CUDA(cudaMemcpyAsync(s->d.cell_box, s->cell_box_host.data(), sizeof(int) * s->ncell, cudaMemcpyHostToDevice,
                          s->stream));
  MW_CUDA(cudaStreamSynchronize(s->stream));
  s->d.ncell = s->ncell;
  s->graph_dirty = true;
  return MW_OK;
}

mw_status alloc_nbr(mw_system* s, int W) {
  dfree(s, s->d.nbr);
  s->d.nbr = nullptr;
  mw_status st;
  if ((st = dalloc(s, &s->d.nbr, (size_t)W * s->N)) != MW_OK) return st;
  MW_CUDA(cudaMemsetAsync(s->d.nbr, 0, sizeof(int) * (size_t)W * s->N, s->stream));
  s->W = s->d.W = W;
  s->list_built = false;
  s->order_ok = false;
  s->graph_dirty = true;
  return MW_OK;
}

void destroy_graphs(mw_system* s) {
  if (s->graph1) cudaGraphExecDestroy(s->graph1);
  if (s->graphK) cudaGraphExecDestroy(s->graphK);
  s->graph1 = s->graphK = nullptr;
}

mw_status set_global_field(mw_system* s, size_t offset, int value) {
  if (value == 0)  // a device-side memset: no host staging of a pageable source
    MW_CUDA(cudaMemsetAsync((char*)s->d.g + offset, 0, sizeof(int), s->stream));
  else
    MW_CUDA(cudaMemcpyAsync((char*)s->d.g + offset, &value, sizeof(int), cudaMemcpyHostToDevice, s->stream));
  return MW_OK;
}

// Applies a pending second half-kick to the stored velocities (before forces
// are recomputed or atoms re-sorted outside a step).
mw_status flush_pending(mw_system* s) {
  if (!s->state_set) return MW_OK;
  k_flush_pending<<<div_up(s->N, kThreads), kThreads, 0, s->stream>>>(s->d);
  MW_CUDA(cudaGetLastError());
  return set_global_field(s, offsetof(Global, pend), 0);
}

mw_status flag_all(mw_system* s) {
  s->order_ok = false;
  k_flag_all<<<div_up(s->nbox, kThreads), kThreads, 0, s->stream>>>(s->d);
  MW_CUDA(cudaGetLastError());
  return MW_OK;
}

mw_status read_global(mw_system* s, Global* g) {
  MW_CUDA(cudaMemcpyAsync(s->gpin(), s->d.g, sizeof(Global), cudaMemcpyDeviceToHost, s->stream));
  MW_CUDA(cudaStreamSynchronize(s->stream));
  *g = *s->gpin();
  return MW_OK;
}

// The last step's thermo records (written on demand by k_record) copied to
// the pinned staging; complete after the next synchronisation of the stream.
mw_status enqueue_thermo(mw_system* s) {
  if (s->record_pending) {
    k_record<<<1, 256, 0, s->stream>>>(s->d);
    MW_CUDA(cudaGetLastError());
    s->record_pending = false;
  }
  MW_CUDA(cudaMemcpyAsync(s->thpin(), s->d.thermo, sizeof(double) * (size_t)s->nbox * TR_N,
                          cudaMemcpyDeviceToHost, s->stream));
  return MW_OK;
}

// The staged records as mw_thermo, one per box.
void unpack_thermo(mw_system* s, mw_thermo* out) {
  const double* t = s->thpin();
  for (int b = 0; b < s->nbox; ++b) {
    const double* r = t + (size_t)b * TR_N;
    mw_thermo& o = out[b];
    o.step = (int64_t)r[TR_STEP];
    o.pe = r[TR_PE];
    o.e2 = r[TR_E2];
    o.e3 = r[TR_E3];
    o.ke = r[TR_KE];
    o.temperature = r[TR_T];
    o.conserved = r[TR_CONS];
    o.pressure = r[TR_P];
    for (int k = 0; k < 6; ++k) o.virial[k] = r[TR_W0 + k];
    o.xi = r[TR_XI];
    o.eta = r[TR_ETA];
    o.rebuilds = (int64_t)r[TR_REBUILDS];
    o.volume = r[TR_VOL];
    for (int k = 0; k < 3; ++k) o.box[k] = r[TR_L0 + k];
  }
}

// After a run's launches: when the caller wants the last record and this
// launch finishes the run, the record is fetched with the status block, in
// one round trip.  *fetched tells whether out holds the run's last record.
mw_status read_global_and_thermo(mw_system* s, Global* g, mw_thermo* out, bool fetch, bool* fetched,
                                 int remaining, unsigned long long step0) {
  mw_status st;
  if (fetch && (st = enqueue_thermo(s)) != MW_OK) return st;
  if ((st = read_global(s, g)) != MW_OK) return st;
  if (fetch) {
    if (g->status == ST_OK && (long long)(g->step - step0) == remaining) {
      unpack_thermo(s, out);
      *fetched = true;
    } else {
      s->record_pending = true;  // the run goes on: the staged record is not its last
    }
  }
  return MW_OK;
}

mw_status status_error(const Global& g) {
  switch (g.status) {
    case ST_GRID: return fail(MW_EGRID, "an isobaric box left its cell grid after step %llu (mw_sync laid the grid out again; continue with mw_step_async)", g.step);
    case ST_OK: return MW_OK;
    case ST_OVERFLOW: return fail(MW_ENLIST_OVERFLOW, "neighbour list overflow (max count %d)", g.max_count);
    case ST_NAN: return fail(MW_ENAN, "non-finite velocity or force at atom slot %d", g.err_index);
    case ST_LOST: return fail(MW_ELOST, "atom slot %d ran away: a velocity component moves it more than a quarter of the shortest box edge per step, or is not finite", g.err_index);
    case ST_TIMEOUT: return fail(MW_ETIMEOUT, "a bounded device-side wait ran out");
    case ST_LEGS: return fail(MW_EINVAL, "more than %d atoms within a*sigma of atom slot %d", kMaxLegsOverflow, g.err_index);
    case ST_CELLS: return fail(MW_ESTATE, "cell counts left by an interrupted run (set a state again)");
    case ST_INPUT: return fail(MW_EINVAL, "non-finite input value of atom %d", g.err_index);
    default: return fail(MW_ECUDA, "device status %d", g.status);
  }
}

// Kernel sequences ----------------------------------------------------------

// The kick kernels: the isobaric instantiations under MW_NPT.
void launch_kick1(mw_system* s, bool cond, cudaGraphConditionalHandle h) {
  const int kb = kick_blocks(s->N, kKThreads);
  const bool npt = s->integ.kind == TH_NPT;
  if (cond)
    npt ? k_kick1<true, true><<<kb, kKThreads, 0, s->stream>>>(s->d, h)
        : k_kick1<true, false><<<kb, kKThreads, 0, s->stream>>>(s->d, h);
  else
    npt ? k_kick1<false, true><<<kb, kKThreads, 0, s->stream>>>(s->d, 0ull)
        : k_kick1<false, false><<<kb, kKThreads, 0, s->stream>>>(s->d, 0ull);
}

void launch_kick2(mw_system* s) {
  const int kb = kick_blocks(s->N, kKThreads, kK2Items);
  if (s->integ.kind == TH_NPT)
    k_kick2<true><<<kb, kKThreads, 0, s->stream>>>(s->d);
  else
    k_kick2<false><<<kb, kKThreads, 0, s->stream>>>(s->d);
}

// Blocks of the two-kernel cell scan: about 512 cells each, at most the
// chunk buffer's capacity.
int scan_blocks(const mw_system* s) { return std::max(1, std::min(s->d.chunk_cap, div_up(s->ncell, 512))); }

void launch_scan(mw_system* s) {
  const int sb = scan_blocks(s);
  k_scan_local<<<sb, kPersThreads, 0, s->stream>>>(s->d);
  k_scan_offsets<<<sb, kPersThreads, 0, s->stream>>>(s->d);
}

void launch_rebuild(mw_system* s) {
  const Dev& d = s->d;
  const int gb = div_up(s->N, kThreads);
  k_bin<<<gb, kThreads, 0, s->stream>>>(d);
  launch_scan(s);
  k_scatter<<<gb, kThreads, 0, s->stream>>>(d);
  k_copyback<<<std::max(gb, div_up(s->nbox, kThreads)), kThreads, 0, s->stream>>>(d);
  k_neigh<<<div_up((long long)s->ncell * 32, kNeighThreads), kNeighThreads, 0, s->stream>>>(d, s->fp.rl2);
}

void launch_force(mw_system* s) {
  const Dev& d = s->d;
  if (s->nsp > 1) {
    const int gb = div_up(s->N, kFAtoms);
    if (s->sp_moment)
      s->count_terms ? k_force_sp<true, 1><<<gb, kFThreads, 0, s->stream>>>(d, s->fp)
                     : k_force_sp<false, 1><<<gb, kFThreads, 0, s->stream>>>(d, s->fp);
    else
      s->count_terms ? k_force_sp<true, 2><<<gb, kFThreads, 0, s->stream>>>(d, s->fp)
                     : k_force_sp<false, 2><<<gb, kFThreads, 0, s->stream>>>(d, s->fp);
    return;
  }
  if (s->engine == MW_ENGINE_PLAIN) {  // the plain path: one thread per atom
    const int gp = div_up(s->N, kPlainThreads);
    if (s->count_terms)
      k_force_plain<true><<<gp, kPlainThreads, 0, s->stream>>>(d, s->fp);
    else
      k_force_plain<false><<<gp, kPlainThreads, 0, s->stream>>>(d, s->fp);
    return;
  }
  const int gb = div_up(s->N, kFThreads / force_shape_lanes(s->force_shape));
#define MW_FORCE_SHAPE(S)                                                                                   \
  case S:                                                                                                  \
    if (s->count_terms)                                                                                    \
      k_force<true, force_shape_lanes(S), force_shape_blocks(S)><<<gb, kFThreads, 0, s->stream>>>(d, s->fp);  \
    else                                                                                                   \
      k_force<false, force_shape_lanes(S), force_shape_blocks(S)><<<gb, kFThreads, 0, s->stream>>>(d, s->fp); \
    break;
  switch (s->force_shape) {
    MW_FORCE_SHAPE(1)
    MW_FORCE_SHAPE(2)
    MW_FORCE_SHAPE(3)
    case 4:  // owner-computes: two passes
      if (s->count_terms) {
        k_force<true, 4, 8, 1><<<gb, kFThreads, 0, s->stream>>>(d, s->fp);
        k_force<true, 4, 8, 2><<<gb, kFThreads, 0, s->stream>>>(d, s->fp);
      } else {
        k_force<false, 4, 8, 1><<<gb, kFThreads, 0, s->stream>>>(d, s->fp);
        k_force<false, 4, 8, 2><<<gb, kFThreads, 0, s->stream>>>(d, s->fp);
      }
      break;
    default:
      MW_FORCE_SHAPE(0)
  }
#undef MW_FORCE_SHAPE
}

// Buffers of the owner-computes force passes (allocated when first selected).
mw_status owner_buffers(mw_system* s) {
  if (s->d.mom) return MW_OK;
  mw_status st;
  if ((st = dalloc(s, &s->d.mom, 3 * (size_t)s->N)) != MW_OK) return st;
  if ((st = dalloc(s, &s->d.legs, (size_t)s->N * kLMax)) != MW_OK) return st;
  if ((st = dalloc(s, &s->d.nleg, (size_t)s->N)) != MW_OK) return st;
  s->graph_dirty = true;  // graphs captured the old Dev
  return MW_OK;
}

// The plain path's steps: every phase kernel launched from the host, step
// after step, no graph (the rebuild kernels return at once on steps without
// a rebuild).
mw_status launch_plain_steps(mw_system* s, int n) {
  for (int k = 0; k < n; ++k) {
    launch_kick1(s, false, 0ull);
    launch_rebuild(s);
    launch_force(s);
    launch_kick2(s);
  }
  MW_CUDA(cudaGetLastError());
  return MW_OK;
}

// One MD step into the stream being captured: kick1, an IF node holding the
// rebuild kernels (condition set on the device by kick1), force, kick2.
mw_status capture_step(mw_system* s) {
  if (std::getenv("MW_GRAPH_NO_CONDITIONAL")) {
    // Same kernels without the IF node (the rebuild kernels return at once
    // when no box needs a rebuild): profilers that skip conditional graphs
    // still see every kernel of the step.
    launch_kick1(s, false, 0ull);
    launch_rebuild(s);
    launch_force(s);
    launch_kick2(s);
    MW_CUDA(cudaGetLastError());
    return MW_OK;
  }
  cudaStreamCaptureStatus cs;
  cudaGraph_t g;
  const cudaGraphNode_t* deps = nullptr;
  size_t nd = 0;
  MW_CUDA(cudaStreamGetCaptureInfo(s->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphConditionalHandle h;
  MW_CUDA(cudaGraphConditionalHandleCreate(&h, g, 0, cudaGraphCondAssignDefault));
  launch_kick1(s, true, h);
  MW_CUDA(cudaGetLastError());
  MW_CUDA(cudaStreamGetCaptureInfo(s->stream, &cs, nullptr, &g, &deps, nullptr, &nd));
  cudaGraphNodeParams p = {};
  p.type = cudaGraphNodeTypeConditional;
  p.conditional.handle = h;
  p.conditional.type = cudaGraphCondTypeIf;
  p.conditional.size = 1;
  cudaGraphNode_t node;
  MW_CUDA(cudaGraphAddNode(&node, g, deps, nullptr, nd, &p));
  MW_CUDA(cudaStreamUpdateCaptureDependencies(s->stream, &node, nullptr, 1, cudaStreamSetCaptureDependencies));
  cudaGraph_t body = p.conditional.phGraph_out[0];
  MW_CUDA(cudaStreamBeginCaptureToGraph(s->cap_stream, body, nullptr, nullptr, 0, cudaStreamCaptureModeThreadLocal));
  cudaStream_t keep = s->stream;
  s->stream = s->cap_stream;
  launch_rebuild(s);
  s->stream = keep;
  MW_CUDA(cudaGetLastError());
  MW_CUDA(cudaStreamEndCapture(s->cap_stream, &body));
  launch_force(s);
  launch_kick2(s);
  MW_CUDA(cudaGetLastError());
  return MW_OK;
}

mw_status set_func_attrs() {
  static bool done = false;
  if (done) return MW_OK;
  mw_status st = persistent_func_attrs();
  if (st != MW_OK) return st;
  done = true;
  return MW_OK;
}

mw_status grow_nbr_after_overflow(mw_system* s, const Global& g) {
  int w = row_width(g.max_count + std::max(8, g.max_count / 4));
  if (w <= s->W) w = row_width(s->W + 1);
  return alloc_nbr(s, w);
}

// Forces (and the thermo snapshot) at the current positions, with overflow recovery.
mw_status ensure_forces(mw_system* s) {
  if (!s->state_set) return fail(MW_ESTATE, "no state set (call mw_set_state first)");
  if (s->forces_valid) return MW_OK;
  mw_status st;
  if ((st = flush_pending(s)) != MW_OK) return st;
  if ((st = set_func_attrs()) != MW_OK) return st;
  for (int attempt = 0; attempt < 4; ++attempt) {
    k_prep_force<<<div_up(std::max(s->N, s->nbox), kThreads), kThreads, 0, s->stream>>>(s->d, 1);
    MW_CUDA(cudaGetLastError());
    launch_rebuild(s);
    launch_force(s);
    if (s->v_pending) {  // velocities of a state just set (their copy ran beside this force call)
      MW_CUDA(cudaStreamWaitEvent(s->stream, s->copy_ev[1], 0));
      k_load_velocities_keep<<<div_up(s->N, kThreads), kThreads, 0, s->stream>>>(s->d, s->d.stage2);
      s->v_pending = false;
    }
    k_thermo_snapshot<<<div_up(s->nbox, kThreads), kThreads, 0, s->stream>>>(s->d);
    MW_CUDA(cudaGetLastError());
    Global g;
    if ((st = read_global(s, &g)) != MW_OK) return st;
    if (s->count_terms) {
      s->npairs = g.npairs / 2;
      s->ntrip = g.ntrip;
    }
    if (g.status == ST_OVERFLOW) {
      if ((st = grow_nbr_after_overflow(s, g)) != MW_OK) return st;
      if ((st = set_global_field(s, offsetof(Global, status), 0)) != MW_OK) return st;
      if ((st = flag_all(s)) != MW_OK) return st;
      continue;
    }
    if (g.status) return status_error(g);
    s->forces_valid = true;
    s->list_built = true;
    s->order_ok = s->integ.kind != TH_NPT;
    s->record_pending = false;  // the snapshot is the newest record
    s->g_known = g;
    s->g_known_valid = true;
    return MW_OK;
  }
  return fail(MW_ENLIST_OVERFLOW, "neighbour list kept overflowing");
}

mw_status capture_graphs(mw_system* s, int ksteps) {
  destroy_graphs(s);
  for (int which = 0; which < 2; ++which) {
    const int steps = which == 0 ? 1 : ksteps;
    cudaGraph_t graph;
    MW_CUDA(cudaStreamBeginCapture(s->stream, cudaStreamCaptureModeThreadLocal));
    mw_status cst = MW_OK;
    for (int k = 0; k < steps && cst == MW_OK; ++k) cst = capture_step(s);
    cudaError_t e = cudaStreamEndCapture(s->stream, &graph);
    if (cst != MW_OK) {
      if (e == cudaSuccess) cudaGraphDestroy(graph);
      return cst;
    }
    if (e != cudaSuccess) return fail(MW_ECUDA, "graph capture failed: %s", cudaGetErrorString(e));
    cudaGraphExec_t ex;
    e = cudaGraphInstantiate(&ex, graph, 0);
    cudaGraphDestroy(graph);
    if (e != cudaSuccess) return fail(MW_ECUDA, "graph instantiate failed: %s", cudaGetErrorString(e));
    (which == 0 ? s->graph1 : s->graphK) = ex;
  }
  s->graphK_steps = ksteps;
  s->graph_dirty = false;
  return MW_OK;
}

// Completes a step interrupted by a neighbour-list overflow (kick1 done).
mw_status finish_interrupted_step(mw_system* s) {
  const int gb = div_up(s->N, kThreads);
  launch_rebuild(s);
  launch_force(s);
  launch_kick2(s);
  MW_CUDA(cudaGetLastError());
  return MW_OK;
}

// An isobaric box left its cell grid (ST_GRID, raised at a step boundary):
// lay the grids out again for the current and coming edges, rebuild every
// box, clear the status.  The run continues from the same step.
mw_status regrid(mw_system* s) {
  s->boxes_stale = true;
  mw_status st;
  int ncell;
  if ((st = layout_cells(s, &ncell)) != MW_OK) {
    s->boxes_stale = true;  // host copy partly rewritten: take the device's again
    return st;
  }
  s->ncell = ncell;
  if ((st = alloc_cells(s)) != MW_OK) return st;
  if ((st = upload_boxes(s)) != MW_OK) return st;
  if ((st = set_global_field(s, offsetof(Global, status), 0)) != MW_OK) return st;
  if ((st = flag_all(s)) != MW_OK) return st;
  s->regrids += 1;
  s->boxes_stale = true;  // the run goes on scaling the boxes
  return MW_OK;
}

// The start-of-step thermostat half is normally computed at the end of the
// previous step; it is recomputed here only after a state or integrator
// change.
mw_status prime_thermostat(mw_system* s) {
  if (s->integ.kind == TH_NPT) {
    s->boxes_stale = true;  // the barostat scales the boxes from here on
    s->order_ok = false;    // and the list positions are no longer in the current boxes
  }
  if (!s->need_prime) return MW_OK;
  k_prime_thermostat<<<div_up(s->nbox, kThreads), kThreads, 0, s->stream>>>(s->d);
  MW_CUDA(cudaGetLastError());
  s->need_prime = false;
  return MW_OK;
}

mw_status run_graph_engine(mw_system* s, int nsteps, mw_thermo* last, bool* fetched, bool plain = false) {
  mw_status st;
  if ((st = prime_thermostat(s)) != MW_OK) return st;
  s->record_pending = true;
  const int K = 16;
  if (!plain && (s->graph_dirty || !s->graph1)) {
    if ((st = capture_graphs(s, K)) != MW_OK) return st;
  }
  int remaining = nsteps;
  int guard = 0;
  int regrid_guard = 0;
  while (remaining > 0) {
    Global g0;
    if (s->g_known_valid) {  // read by ensure_forces just before, nothing run since
      g0 = s->g_known;
      s->g_known_valid = false;
    } else if ((st = read_global(s, &g0)) != MW_OK) {
      return st;
    }
    if (g0.status == ST_GRID) {
      if (++regrid_guard > 8) return fail(MW_EGRID, "cell grid of an isobaric box kept failing");
      if ((st = regrid(s)) != MW_OK) return st;
      if (!plain && (st = capture_graphs(s, K)) != MW_OK) return st;
      continue;
    }
    const unsigned long long step0 = g0.step;
    if (plain) {
      if ((st = launch_plain_steps(s, remaining)) != MW_OK) return st;
    } else {
      const int full = remaining / K, rest = remaining % K;
      for (int k = 0; k < full; ++k) MW_CUDA(cudaGraphLaunch(s->graphK, s->stream));
      for (int k = 0; k < rest; ++k) MW_CUDA(cudaGraphLaunch(s->graph1, s->stream));
    }
    Global g;
    if ((st = read_global_and_thermo(s, &g, last, last != nullptr, fetched, remaining, step0)) != MW_OK) return st;
    const int done = (int)(g.step - step0);
    s->host_step += done;
    if (g.status == ST_OVERFLOW) {
      if (++guard > 8) return fail(MW_ENLIST_OVERFLOW, "neighbour list kept overflowing");
      if ((st = grow_nbr_after_overflow(s, g)) != MW_OK) return st;
      if ((st = set_global_field(s, offsetof(Global, status), 0)) != MW_OK) return st;
      if ((st = flag_all(s)) != MW_OK) return st;
      if ((st = finish_interrupted_step(s)) != MW_OK) return st;
      Global g2;
      if ((st = read_global(s, &g2)) != MW_OK) return st;
      if (g2.status == ST_OVERFLOW) continue;  // grow again, same step
      if (g2.status) return status_error(g2);
      s->host_step += 1;
      remaining -= done + 1;
      if (!plain && (st = capture_graphs(s, K)) != MW_OK) return st;
      continue;
    }
    if (g.status == ST_GRID) {  // stopped at a step boundary; the loop head lays the grid out again
      remaining -= done;
      if (done > 0) regrid_guard = 0;
      continue;
    }
    if (g.status) return status_error(g);
    remaining -= done;
    if (done == 0) return fail(MW_ECUDA, "no progress in graph engine");
  }
  return MW_OK;
}

// The device-side address of page-locked host memory (cudaMallocHost,
// cudaHostAlloc, cudaHostRegister), through which kernels read it in place;
// null for pageable memory.
const double* mapped_host(const double* p) {
  cudaPointerAttributes a{};
  if (cudaPointerGetAttributes(&a, p) != cudaSuccess) {
    cudaGetLastError();  // clear the error of an unknown pointer
    return nullptr;
  }
  if (a.type != cudaMemoryTypeHost || !a.devicePointer) return nullptr;
  return static_cast<const double*>(a.devicePointer);
}

// The copy stream and its events (created on first use).
mw_status copy_lane(mw_system* s) {
  if (!s->copy_stream) MW_CUDA(cudaStreamCreateWithFlags(&s->copy_stream, cudaStreamNonBlocking));
  for (auto& e : s->copy_ev)
    if (!e) MW_CUDA(cudaEventCreateWithFlags(&e, cudaEventDisableTiming));
  return MW_OK;
}

mw_status ensure_forces(mw_system* s);

// mw_set_state in the kept order with host velocities: the positions are
// copied and loaded, and the force call at them (which the next step or
// energy call would make) runs while the velocities are copied in on the
// copy stream; the velocities are then loaded before the thermo snapshot.
// A non-finite input refuses the state as in the other paths.
mw_status set_state_keep_overlapped(mw_system* s, const double* x, const double* v, size_t bytes) {
  mw_status st;
  if ((st = copy_lane(s)) != MW_OK) return st;
  // the positions first, alone on the link; the velocities after them (one
  // copy fills the link in each direction, two would share it)
  MW_CUDA(cudaMemcpyAsync(s->d.stage, x, bytes, cudaMemcpyHostToDevice, s->stream));
  MW_CUDA(cudaEventRecord(s->copy_ev[0], s->stream));  // (earlier work on the staging buffers is done too)
  MW_CUDA(cudaStreamWaitEvent(s->copy_stream, s->copy_ev[0], 0));
  MW_CUDA(cudaMemcpyAsync(s->d.stage2, v, bytes, cudaMemcpyHostToDevice, s->copy_stream));
  MW_CUDA(cudaEventRecord(s->copy_ev[1], s->copy_stream));
  MW_CUDA(cudaMemsetAsync(s->d.bst, 0, sizeof(BoxState) * s->nbox, s->stream));
  const size_t mc = offsetof(Global, max_count);
  MW_CUDA(cudaMemsetAsync(s->d.g, 0, mc, s->stream));
  MW_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(s->d.g) + mc + sizeof(int), 0, sizeof(Global) - mc - sizeof(int),
                          s->stream));
  const int gl = div_up(std::max(std::max(s->N, s->ncell), s->nbox), kThreads);
  k_load_positions_keep<<<gl, kThreads, 0, s->stream>>>(s->d, s->d.stage, s->count_terms,
                                                         (float)(0.25 * s->skin * s->skin));
  MW_CUDA(cudaGetLastError());
  s->v_pending = true;
  s->state_set = true;
  s->forces_valid = false;
  s->need_prime = true;  // thermostat at rest: xi = eta = 0, KE of the new velocities
  s->host_step = 0;
  st = ensure_forces(s);
  if (s->v_pending) {  // (the force call stopped before loading them)
    cudaStreamSynchronize(s->copy_stream);
    s->v_pending = false;
    if (st == MW_OK) st = fail(MW_ECUDA, "velocities not loaded");
  }
  if (st != MW_OK) {
    Global gh;
    const bool input = read_global(s, &gh) == MW_OK && gh.status == ST_INPUT;
    s->state_set = false;  // the arrays hold part of a refused state
    s->order_ok = false;
    s->forces_valid = false;
    if (input) return fail(MW_EINVAL, "non-finite position or velocity of atom %d", gh.err_index);
    return st;
  }
  return MW_OK;
}

mw_status do_set_state(mw_system* s, const double* x, const double* v, bool dev) {
  if (!s) return fail(MW_EINVAL, "system is NULL");
  if (!x) return fail(MW_EINVAL, "positions are NULL");
  const size_t bytes = sizeof(double) * 3 * (size_t)s->N;
  const double* xd = x;
  const double* vd = v;
  const bool keep = s->state_set && s->order_ok && s->integ.kind != TH_NPT;
  if (!dev && keep && v) return set_state_keep_overlapped(s, x, v, bytes);
  if (!dev && keep) {
    // the current order is kept, so the loading kernel reads the inputs
    // through the atom permutation: one copy of each array to device memory
    // first (a DMA at the link's rate) instead of scattered reads of host
    // memory
    MW_CUDA(cudaMemcpyAsync(s->d.stage, x, bytes, cudaMemcpyHostToDevice, s->stream));
    xd = s->d.stage;
    if (v) {
      MW_CUDA(cudaMemcpyAsync(s->d.stage2, v, bytes, cudaMemcpyHostToDevice, s->stream));
      vd = s->d.stage2;
    }
  } else if (!dev) {  // (finiteness is checked on the device, as for device inputs)
    // pinned (page-locked) host arrays are read by k_load_state in place,
    // through their device mapping; pageable ones are copied to staging first
    const double* xm = mapped_host(x);
    if (xm) {
      xd = xm;
    } else {
      MW_CUDA(cudaMemcpyAsync(s->d.stage, x, bytes, cudaMemcpyHostToDevice, s->stream));
      xd = s->d.stage;
    }
    if (v) {
      const double* vm = mapped_host(v);
      if (vm) {
        vd = vm;
      } else {
        MW_CUDA(cudaMemcpyAsync(s->d.stage2, v, bytes, cudaMemcpyHostToDevice, s->stream));
        vd = s->d.stage2;
      }
    }
  }
  // reset thermostat / accumulators / counters: zeroed here, the non-zero
  // starting values set by the loading kernel
  MW_CUDA(cudaMemsetAsync(s->d.bst, 0, sizeof(BoxState) * s->nbox, s->stream));
  // one pass over atoms and cells; the cell counts start from zero (a run
  // that stopped on an error may have binned atoms without the scan that
  // clears them)
  const int gl = div_up(std::max(std::max(s->N, s->ncell), s->nbox), kThreads);
  if (keep) {
    // the current order and lists stay (boxes whose atoms moved more than
    // half the skin from their list positions are flagged for a rebuild);
    // the widest-row record of those lists is kept
    const size_t mc = offsetof(Global, max_count);
    MW_CUDA(cudaMemsetAsync(s->d.g, 0, mc, s->stream));
    MW_CUDA(cudaMemsetAsync(reinterpret_cast<char*>(s->d.g) + mc + sizeof(int), 0, sizeof(Global) - mc - sizeof(int),
                            s->stream));
    k_load_state_keep<<<gl, kThreads, 0, s->stream>>>(s->d, xd, vd, s->count_terms,
                                                      (float)(0.25 * s->skin * s->skin));
  } else {
    MW_CUDA(cudaMemsetAsync(s->d.g, 0, sizeof(Global), s->stream));
    k_load_state<<<gl, kThreads, 0, s->stream>>>(s->d, xd, vd, s->boxid, s->count_terms);
  }
  MW_CUDA(cudaGetLastError());
  Global gh;
  mw_status st;
  if ((st = read_global(s, &gh)) != MW_OK) return st;
  if (gh.status == ST_INPUT) {
    s->state_set = false;  // the arrays hold part of a refused state
    s->order_ok = false;
    return fail(MW_EINVAL, "non-finite position or velocity of atom %d", gh.err_index);
  }
  if (!keep) s->order_ok = false;  // identity order: sorted and listed by the next force call
  s->state_set = true;
  s->forces_valid = false;
  s->need_prime = true;  // thermostat at rest: xi = eta = 0, KE of the new velocities
  s->host_step = 0;
  return MW_OK;
}

mw_status validate_integ(mw_system* s, const mw_integrator* in) {
  if (!in) return fail(MW_EINVAL, "integrator is NULL");
  if (!(in->dt > 0) || !std::isfinite(in->dt)) return fail(MW_EINVAL, "dt must be > 0");
  if (in->thermostat < MW_NVE || in->thermostat > MW_NPT) return fail(MW_EINVAL, "unknown thermostat");
  if (in->thermostat != MW_NVE && !(in->tau > 0)) return fail(MW_EINVAL, "tau must be > 0");
  const bool npt = in->thermostat == MW_NPT;
  if (npt && (!(in->tau_p > 0) || !std::isfinite(in->tau_p) || !std::isfinite(in->p_ext)))
    return fail(MW_EINVAL, "isobaric runs need tau_p > 0 and a finite p_ext");
  mw_status st;
  if ((st = pull_boxes(s)) != MW_OK) return st;
  bool boxes_changed = false;
  for (int b = 0; b < s->nbox; ++b) {
    const double T0 = in->T0_per_box ? in->T0_per_box[b] : in->T0;
    if (in->thermostat != MW_NVE && !(T0 > 0)) return fail(MW_EINVAL, "T0 must be > 0");
    Box& bx = s->boxes[b];
    const double Q = bx.Ndf * kKB * T0 * in->tau * in->tau;
    const double q4 = 0.25 * in->dt / Q;
    if (bx.T0 != T0 || bx.Q != Q || bx.q4 != q4) {
      bx.T0 = T0;
      bx.Q = Q;
      bx.invQ = 1.0 / Q;
      bx.ndfkT0 = bx.Ndf * kKB * T0;
      bx.q4 = q4;
      bx.q4f = (float)q4;
      boxes_changed = true;
    }
    if (npt) {
      const double a3 = 1.0 + 3.0 / bx.Ndf;
      const double W = (bx.Ndf + 3.0) * kKB * T0 * in->tau_p * in->tau_p;
      if (bx.a3 != (float)a3 || bx.W != W) {
        bx.a3 = (float)a3;
        bx.W = W;
        boxes_changed = true;
      }
    }
    for (int k = 0; k < 3; ++k) {
      const double dtL = in->dt / bx.L[k];
      if (npt) {  // the drift factor of an isobaric step is set on the device (barostat start half)
        bx.dtL[k] = dtL;
        continue;
      }
      const float dtL64 = (float)std::ldexp(dtL, 64);
      if (bx.dtL[k] != dtL || bx.dtL64[k] != dtL64) {
        bx.dtL[k] = dtL;
        bx.dtL64[k] = dtL64;
        boxes_changed = true;
      }
    }
    // a velocity component of magnitude >= 2^floor(log2(lost / dt)) (between
    // lost/(2 dt) and lost/dt) moves an atom at least a quarter of the
    // shortest edge in one step: the run is reported as lost (FP32 exponent)
    const int ve = std::min(255, std::max(1, 127 + (int)std::floor(std::log2((double)bx.lost / in->dt))));
    if (bx.vexp_lost != ve) {
      bx.vexp_lost = ve;
      boxes_changed = true;
    }
  }
  Integ I{};
  I.dt = in->dt;
  I.cf = 0.5 * in->dt * kFCONV / s->mass;
  I.cf_f = (float)I.cf;
  I.ke_fac = 0.5 * s->mass / kFCONV;
  I.tau = in->thermostat == MW_NVE ? 1.0 : in->tau;
  I.kind = in->thermostat;
  I.half_skin2 = (float)(0.25 * s->skin * s->skin);
  I.p_ext = npt ? in->p_ext / kATM : 0.0;
  I.skin = (float)s->skin;
  I.rlist = (float)r_list(s);
  const bool integ_changed = std::memcmp(&I, &s->integ, sizeof I) != 0;
  if ((boxes_changed || integ_changed) && s->state_set) {
    // the pending half-kick belongs to the old integrator (the last step's
    // end half was taken with it too); the start half is redone with the new
    if ((st = flush_pending(s)) != MW_OK) return st;
  }
  if (boxes_changed && (st = upload_boxes(s)) != MW_OK) return st;
  if (integ_changed) {
    if ((I.kind == TH_NPT) != (s->integ.kind == TH_NPT)) s->graph_dirty = true;  // other kick kernels
    s->integ = I;
    if ((st = upload_integ(s)) != MW_OK) return st;
  }
  if (boxes_changed || integ_changed) s->need_prime = true;
  return MW_OK;
}

mw_status create_common(mw_system** out, int nbox, const int* n, const double* box, const mw_params* prm,
                        double mass, double skin, void* stream) {
  if (!out) return fail(MW_EINVAL, "out is NULL");
  *out = nullptr;
  if (nbox < 1 || !n || !box) return fail(MW_EINVAL, "need nbox >= 1, n and box");
  mw_status st;
  if ((st = check_params(prm)) != MW_OK) return st;
  if (!(mass > 0) || !(skin >= 0) || !std::isfinite(mass) || !std::isfinite(skin))
    return fail(MW_EINVAL, "mass must be > 0 and skin >= 0");
  long long total = 0;
  for (int b = 0; b < nbox; ++b) {
    if (n[b] < 2) return fail(MW_EINVAL, "box %d has %d atoms (need >= 2)", b, n[b]);
    for (int k = 0; k < 3; ++k)
      if (!(box[3 * b + k] > 0) || !std::isfinite(box[3 * b + k])) return fail(MW_EINVAL, "bad box edge");
    total += n[b];
  }
  if (total > (1ll << 28)) return fail(MW_EINVAL, "too many atoms (%lld)", total);
  mw_system* s = new mw_system();
  {
    const size_t pin = mw_system::kPinThermoOff + sizeof(double) * (size_t)nbox * TR_N;
    cudaError_t e = cudaMallocHost(&s->hpin, pin);
    if (e != cudaSuccess) {
      delete s;
      return fail(MW_ENOMEM, "cudaMallocHost of %zu bytes failed: %s", pin, cudaGetErrorString(e));
    }
  }
  s->nbox = nbox;
  s->N = (int)total;
  s->prm = *prm;
  s->mass = mass;
  s->skin = skin;
  s->stream = (cudaStream_t)stream;
  if (!s->stream) {
    cudaError_t e = cudaStreamCreateWithFlags(&s->stream, cudaStreamNonBlocking);
    if (e != cudaSuccess) {
      cudaFreeHost(s->hpin);
      delete s;
      return fail(MW_ECUDA, "cudaStreamCreate failed: %s", cudaGetErrorString(e));
    }
    s->own_stream = true;
  }
  if (cudaStreamCreateWithFlags(&s->cap_stream, cudaStreamNonBlocking) != cudaSuccess) {
    if (s->own_stream) cudaStreamDestroy(s->stream);
    cudaFreeHost(s->hpin);
    delete s;
    return fail(MW_ECUDA, "cudaStreamCreate failed");
  }
  s->n.assign(n, n + nbox);
  s->off.resize(nbox);
  s->boxes.resize(nbox);
  int o = 0;
  for (int b = 0; b < nbox; ++b) {
    Box& bx = s->boxes[b];
    std::memset(&bx, 0, sizeof bx);
    for (int k = 0; k < 3; ++k) {
      bx.L[k] = box[3 * b + k];
      bx.qs[k] = 4294967296.0 / bx.L[k];
      bx.Lq[k] = (float)(bx.L[k] / 4294967296.0);
    }
    bx.lost = (float)(0.5 * std::min(bx.L[0], std::min(bx.L[1], bx.L[2])));
    bx.off = o;
    bx.n = n[b];
    bx.Ndf = 3.0 * n[b] - 3.0;
    bx.T0 = 0;
    bx.Q = 1;
    bx.invQ = 1;
    bx.vexp_lost = 255;
    bx.volume = bx.L[0] * bx.L[1] * bx.L[2];
    bx.inv_ndf_kb = bx.Ndf > 0 ? 1.0 / (bx.Ndf * kKB) : 0.0;
    bx.p_fac = kATM / (3.0 * bx.volume);
    s->off[b] = o;
    o += n[b];
  }
  make_fparams(s);
  if ((st = layout_cells(s, &s->ncell)) != MW_OK) {
    if (s->own_stream) cudaStreamDestroy(s->stream);
    cudaStreamDestroy(s->cap_stream);
    cudaFreeHost(s->hpin);
    delete s;
    return st;
  }
  auto bad = [&](mw_status e) {
    mw_system_destroy(s);
    return e;
  };
  const size_t N = s->N;
  Dev& d = s->d;
  d.N = s->N;
  d.nbox = nbox;
  unsigned long long** pos[] = {&d.x, &d.y, &d.z, &d.tx, &d.ty, &d.tz};
  for (unsigned long long** p : pos)
    if ((st = dalloc(s, p, N)) != MW_OK) return bad(st);
  float2** vel[] = {&d.vx, &d.vy, &d.vz, &d.tvx, &d.tvy, &d.tvz};
  for (float2** p : vel)
    if ((st = dalloc(s, p, N)) != MW_OK) return bad(st);
  if ((st = dalloc(s, &d.img, N)) != MW_OK || (st = dalloc(s, &d.timg, N)) != MW_OK) return bad(st);
  if ((st = dalloc(s, &d.q, N)) != MW_OK || (st = dalloc(s, &d.qb, N)) != MW_OK ||
      (st = dalloc(s, &d.tq, N)) != MW_OK || (st = dalloc(s, &d.f, N)) != MW_OK ||
      (st = dalloc(s, &d.id, N)) != MW_OK || (st = dalloc(s, &d.tid, N)) != MW_OK ||
      (st = dalloc(s, &d.cell, N)) != MW_OK || (st = dalloc(s, &d.rank, N)) != MW_OK ||
      (st = dalloc(s, &d.nbr_cnt, N)) != MW_OK || (st = dalloc(s, &d.over, N)) != MW_OK ||
      (st = dalloc(s, &d.stage, 3 * N)) != MW_OK || (st = dalloc(s, &d.stage2, 3 * N)) != MW_OK ||
      (st = dalloc(s, &s->boxid, N)) != MW_OK || (st = dalloc(s, &s->eout, 9 * (size_t)nbox)) != MW_OK ||
      (st = dalloc(s, &d.chunk, 4096)) != MW_OK)
    return bad(st);
  d.chunk_cap = 4096;
  if (cudaMemsetAsync(d.nbr_cnt, 0, sizeof(int) * N, s->stream) != cudaSuccess)
    return bad(fail(MW_ECUDA, "memset failed"));
  Box* dbox = nullptr;
  BoxState* dbst = nullptr;
  double* dth = nullptr;
  Global* dg = nullptr;
  Integ* dint = nullptr;
  if ((st = dalloc(s, &dbox, nbox)) != MW_OK || (st = dalloc(s, &dbst, nbox)) != MW_OK ||
      (st = dalloc(s, &dth, (size_t)nbox * TR_N)) != MW_OK || (st = dalloc(s, &dg, 1)) != MW_OK ||
      (st = dalloc(s, &dint, 1)) != MW_OK)
    return bad(st);
  d.box = dbox;
  d.bst = dbst;
  d.thermo = dth;
  d.g = dg;
  d.integ = dint;
  if ((st = alloc_cells(s)) != MW_OK) return bad(st);
  if ((st = alloc_nbr(s, initial_width(s))) != MW_OK) return bad(st);
  if ((st = adjoint_alloc(s)) != MW_OK) return bad(st);
  std::vector<int> bid(N);
  for (int b = 0; b < nbox; ++b)
    for (int k = 0; k < n[b]; ++k) bid[s->off[b] + k] = b;
  cudaError_t e = cudaMemcpyAsync(s->boxid, bid.data(), sizeof(int) * N, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return bad(fail(MW_ECUDA, "upload failed: %s", cudaGetErrorString(e)));
  if ((st = upload_boxes(s)) != MW_OK) return bad(st);
  s->integ.dt = 0;
  s->integ.cf = 0;
  s->integ.ke_fac = 0.5 * s->mass / kFCONV;
  s->integ.tau = 1;
  s->integ.kind = TH_NVE;
  s->integ.half_skin2 = (float)(0.25 * skin * skin);
  s->integ.skin = (float)skin;
  s->integ.rlist = (float)r_list(s);
  if ((st = upload_integ(s)) != MW_OK) return bad(st);
  Global g{};
  e = cudaMemcpyAsync(d.g, &g, sizeof g, cudaMemcpyHostToDevice, s->stream);
  if (e != cudaSuccess) return bad(fail(MW_ECUDA, "upload failed: %s", cudaGetErrorString(e)));
  e = cudaStreamSynchronize(s->stream);
  if (e != cudaSuccess) return bad(fail(MW_ECUDA, "sync failed: %s", cudaGetErrorString(e)));
  *out = s;
  return MW_OK;
}

}  // namespace

#include "mw_persistent_host.inc"
#include "mw_adjoint_host.inc"
#include "mw_autotune.inc"
#include "mw_structure_host.inc"
#include "mw_checkpoint_host.inc"

extern "C" {

const char* mw_last_error(void) { return g_err.c_str(); }

mw_status mw_params_default(mw_params* out) {
  if (!out) return fail(MW_EINVAL, "out is NULL");
  // Sec. II.A (SW form: A, B, p, q, gamma, a, theta0) and Sec. II.D (mW: lambda, epsilon, sigma)
  out->lambda = 23.15;
  out->epsilon = 6.189;
  out->sigma = 2.3925;
  out->a = 1.8;
  out->gamma = 1.2;
  out->A = 7.049556277;
  out->B = 0.6022245584;
  out->cos_theta0 = -1.0 / 3.0;
  out->p = 4;
  out->q = 0;
  return MW_OK;
}

mw_status mw_system_create(mw_system** out, int n, const double box[3], const mw_params* prm, double mass,
                           double skin, void* stream) {
  return create_common(out, 1, &n, box, prm, mass, skin, stream);
}

mw_status mw_batch_create(mw_system** out, int nbox, const int* n, const double* box, const mw_params* prm,
                          double mass, double skin, void* stream) {
  return create_common(out, nbox, n, box, prm, mass, skin, stream);
}

mw_status mw_system_destroy(mw_system* s) {
  if (!s) return MW_OK;
  if (s->stream || true) cudaStreamSynchronize(s->stream);
  destroy_graphs(s);
  for (void* p : s->allocs) cudaFree(p);
  if (s->own_stream) cudaStreamDestroy(s->stream);
  if (s->cap_stream) cudaStreamDestroy(s->cap_stream);
  if (s->copy_stream) cudaStreamDestroy(s->copy_stream);
  for (auto e : s->copy_ev)
    if (e) cudaEventDestroy(e);
  if (s->hpin) cudaFreeHost(s->hpin);
  delete s;
  return MW_OK;
}

mw_status mw_set_state(mw_system* s, const double* x, const double* v) {
  Range range_("mw_set_state");
  return do_set_state(s, x, v, false);
}

mw_status mw_set_state_dev(mw_system* s, const double* x_dev, const double* v_dev) {
  return do_set_state(s, x_dev, v_dev, true);
}

mw_status mw_get_state(mw_system* s, double* x, double* v) {
  if (!s) return fail(MW_EINVAL, "system is NULL");
  if (!s->state_set) return fail(MW_ESTATE, "no state set");
  const size_t bytes = sizeof(double) * 3 * (size_t)s->N;
  k_gather_state<<<div_up(s->N, kThreads), kThreads, 0, s->stream>>>(s->d, x ? s->d.stage : nullptr,
                                                                     v ? s->d.stage2 : nullptr, 0);
  MW_CUDA(cudaGetLastError());
  if (x) MW_CUDA(cudaMemcpyAsync(x, s->d.stage, bytes, cudaMemcpyDeviceToHost, s->stream));
  if (v) MW_CUDA(cudaMemcpyAsync(v, s->d.stage2, bytes, cudaMemcpyDeviceToHost, s->stream));
  MW_CUDA(cudaStreamSynchronize(s->stream));
  return MW_OK;
}

mw_status mw_get_unwrapped(mw_system* s, double* x) {
  if (!s || !x) return fail(MW_EINVAL, "bad arguments");
  if (!s->state_set) return fail(MW_ESTATE, "no state set");
  const size_t bytes = sizeof(double) * 3 * (size_t)s->N;
  k_gather_state<<<div_up(s->N, kThreads), kThreads, 0, s->stream>>>(s->d, s->d.stage, nullptr, 1);
  MW_CUDA(cudaGetLastError());
  MW_CUDA(cudaMemcpyAsync(x, s->d.stage, bytes, cudaMemcpyDeviceToHost, s->stream));
  MW_CUDA(cudaStreamSynchronize(s->stream));
  return MW_OK;
}

mw_status mw_get_state_dev(mw_system* s, double* x_dev, double* v_dev) {
  if (!s) return fail(MW_EINVAL, "system is NULL");
  if (!s->state_set) return fail(MW_ESTATE, "no state set");
  k_gather_state<<<div_up(s->N, kThreads), kThreads, 0, s->stream>>>(s->d, x_dev, v_dev, 0);
  MW_CUDA(cudaGetLastError());
  MW_CUDA(cudaStreamSynchronize(s->stream));
  return MW_OK;
}

mw_status mw_set_params(mw_system* s, const mw_params* prm) {
  if (!s) return fail(MW_EINVAL, "system is NULL");
  mw_status st;
  if ((st = check_params(prm)) != MW_OK) return st;
  if ((st = flush_pending(s)) != MW_OK) return st;  // the pending half-kick belongs to the old potential
  const mw_params old = s->prm;
  const int old_nsp = s->nsp;
  s->prm = *prm;
  s->nsp = 1;  // one species again
  int ncell;
  if ((st = layout_cells(s, &ncell)) != MW_OK) {
    s->prm = old;
    s->nsp = old_nsp;
    layout_cells(s, &ncell);
    return st;
  }
  s->d.nsp = 1;
  s->d.typ = nullptr;
  make_fparams(s);
  s->ncell = ncell;
  if ((st = alloc_cells(s)) != MW_OK) return st;
  if ((st = upload_boxes(s)) != MW_OK) return st;
  s->graph_dirty = true;
  s->forces_valid = false;
  if (s->state_set) {
    if ((st = flag_all(s)) != MW_OK) return st;
  }
  MW_CUDA(cudaStreamSynchronize(s->stream));
  return MW_OK;
}

mw_status mw_set_species(mw_system* s, int nt, const mw_params* table, const int* types) {
  Range range_("mw_set_species");
  if (!s) return fail(MW_EINVAL, "system is NULL");
  if (nt < 1 || nt > MW_MAX_SPECIES) return fail(MW_EINVAL, "need 1 <= nt <= %d species", MW_MAX_SPECIES);
  if (!table) return fail(MW_EINVAL, "table is NULL");
  if (nt == 1) return mw_set_params(s, &table[0]);
  if (!types) return fail(MW_EINVAL, "types is NULL");
  if (s->engine == MW_ENGINE_PLAIN) return fail(MW_EINVAL, "the plain engine has one species only");
  mw_status st;
  const size_t ne = (size_t)nt * nt * nt;
  auto E = [&](int a, int b, int c) -> const mw_params& { return table[((size_t)a * nt + b) * nt + c]; };
  for (size_t k = 0; k < ne; ++k)
    if ((st = check_params(&table[k])) != MW_OK) return st;
  double rcmax = 0;
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      const mw_params& ab = E(a, b, b);
      const mw_params& ba = E(b, a, a);
      if (ab.epsilon != ba.epsilon || ab.sigma != ba.sigma || ab.a != ba.a || ab.A != ba.A || ab.B != ba.B ||
          ab.p != ba.p || ab.q != ba.q)
        return fail(MW_EINVAL, "pair entries (%d,%d,%d) and (%d,%d,%d) differ in a two-body parameter", a, b, b,
                    b, a, a);
      rcmax = std::max(rcmax, ab.a * ab.sigma);
      for (int c = 0; c < nt; ++c) {
        const mw_params& abc = E(a, b, c);
        const mw_params& acb = E(a, c, b);
        if (abc.lambda != acb.lambda || abc.epsilon != acb.epsilon || abc.cos_theta0 != acb.cos_theta0)
          return fail(MW_EINVAL, "entries (%d,%d,%d) and (%d,%d,%d) differ in lambda, epsilon or cos_theta0", a,
                      b, c, a, c, b);
      }
    }
  for (int i = 0; i < s->N; ++i)
    if (types[i] < 0 || types[i] >= nt) return fail(MW_EINVAL, "types[%d] = %d is outside [0, %d)", i, types[i], nt);
  // FP32 constants of every pair and triplet
  const double l2e = 1.4426950408889634;
  std::vector<SpPair> pairs((size_t)nt * nt);
  std::vector<float2> tri(ne);
  for (int a = 0; a < nt; ++a)
    for (int b = 0; b < nt; ++b) {
      const mw_params& p = E(a, b, b);
      SpPair& q = pairs[(size_t)a * nt + b];
      const double rc = p.a * p.sigma;
      q.rc = (float)rc;
      q.rc2 = (float)(rc * rc);
      q.sig = (float)p.sigma;
      q.sig_l2e = (float)(p.sigma * l2e);
      q.gsig = (float)(p.gamma * p.sigma);
      q.gsig_l2e = (float)(p.gamma * p.sigma * l2e);
      q.Aeps = (float)(p.A * p.epsilon);
      q.B = (float)p.B;
      q.p = p.p;
      q.q = p.q;
      q.rc_lo = (float)(rc - (double)q.rc);
      q.sig_lo = (float)(p.sigma - (double)q.sig);
      q.sig_l2e_lo = (float)(p.sigma * l2e - (double)q.sig_l2e);
      q.gsig_l2e_lo = (float)(p.gamma * p.sigma * l2e - (double)q.gsig_l2e);
      q.B_lo = (float)(p.B - (double)q.B);
      q.h = (float)std::sqrt(std::max(0.0, E(a, b, b).lambda * E(a, b, b).epsilon));
      q.c0 = (float)E(a, 0, 0).cos_theta0;
      for (int c = 0; c < nt; ++c) {
        const mw_params& t = E(a, b, c);
        tri[((size_t)a * nt + b) * nt + c] = make_float2((float)(t.lambda * t.epsilon), (float)t.cos_theta0);
      }
    }
  // moment kernel when lambda epsilon of (a; b, c) = h_ab h_ac (to 1e-9) and
  // cos theta0 is the centre's
  bool moment = true;
  for (int a = 0; a < nt && moment; ++a)
    for (int b = 0; b < nt && moment; ++b)
      for (int c = 0; c < nt && moment; ++c) {
        const mw_params& t = E(a, b, c);
        const double le = t.lambda * t.epsilon;
        const double hh = std::sqrt(E(a, b, b).lambda * E(a, b, b).epsilon * E(a, c, c).lambda * E(a, c, c).epsilon);
        if (t.cos_theta0 != E(a, 0, 0).cos_theta0 || std::fabs(le - hh) > 1e-9 * std::max(le, hh)) moment = false;
      }
  if ((st = flush_pending(s)) != MW_OK) return st;  // the pending half-kick belongs to the old potential
  if (!s->typ_buf) {
    if ((st = dalloc(s, &s->typ_buf, s->N)) != MW_OK || (st = dalloc(s, &s->ttyp_buf, s->N)) != MW_OK ||
        (st = dalloc(s, &s->utyp_buf, s->N)) != MW_OK ||
        (st = dalloc(s, &s->sp_pair_buf, (size_t)kMaxSpecies * kMaxSpecies)) != MW_OK ||
        (st = dalloc(s, &s->sp_tri_buf, (size_t)kMaxSpecies * kMaxSpecies * kMaxSpecies)) != MW_OK)
      return st;
  }
  MW_CUDA(cudaMemcpyAsync(s->sp_pair_buf, pairs.data(), sizeof(SpPair) * pairs.size(), cudaMemcpyHostToDevice,
                          s->stream));
  MW_CUDA(cudaMemcpyAsync(s->sp_tri_buf, tri.data(), sizeof(float2) * tri.size(), cudaMemcpyHostToDevice, s->stream));
  MW_CUDA(cudaMemcpyAsync(s->utyp_buf, types, sizeof(int) * s->N, cudaMemcpyHostToDevice, s->stream));
  const int old_nsp = s->nsp;
  const double old_rc = s->sp_rc_max;
  s->nsp = nt;
  s->sp_rc_max = rcmax;
  int ncell;
  if ((st = layout_cells(s, &ncell)) != MW_OK) {
    s->nsp = old_nsp;
    s->sp_rc_max = old_rc;
    layout_cells(s, &ncell);
    return st;
  }
  s->sp_table.assign(table, table + ne);
  s->sp_moment = moment;
  s->d.nsp = nt;
  s->d.typ = s->typ_buf;
  s->d.ttyp = s->ttyp_buf;
  s->d.utyp = s->utyp_buf;
  s->d.sp_pair = s->sp_pair_buf;
  s->d.sp_tri = s->sp_tri_buf;
  make_fparams(s);
  s->ncell = ncell;
  if ((st = alloc_cells(s)) != MW_OK) return st;
  if ((st = upload_boxes(s)) != MW_OK) return st;
  const int w = initial_width(s);
  if (w > s->W && (st = alloc_nbr(s, w)) != MW_OK) return st;
  s->graph_dirty = true;
  s->forces_valid = false;
  if (s->state_set) {
    k_gather_types<<<div_up(s->N, kThreads), kThreads, 0, s->stream>>>(s->d);
    MW_CUDA(cudaGetLastError());
    if ((st = flag_all(s)) != MW_OK) return st;
  }
  MW_CUDA(cudaStreamSynchronize(s->stream));
  return MW_OK;
}

mw_status mw_build_neighbors(mw_system* s, int* max_count_out) {
  Range range_("mw_build_neighbors");
  if (!s) return fail(MW_EINVAL, "system is NULL");
  if (!s->state_set) return fail(MW_ESTATE, "no state set");
  mw_status st;
  if ((st = flush_pending(s)) != MW_OK) return st;  // atoms get re-sorted, forces do not follow
  for (int attempt = 0; attempt < 4; ++attempt) {
    if ((st = flag_all(s)) != MW_OK) return st;
    launch_rebuild(s);
    k_prep_force<<<div_up(s->nbox, kThreads), kThreads, 0, s->stream>>>(s->d, 0);  // list consumed
    MW_CUDA(cudaGetLastError());
    Global g;
    if ((st = read_global(s, &g)) != MW_OK) return st;
    if (g.status == ST_OVERFLOW) {
      if ((st = grow_nbr_after_overflow(s, g)) != MW_OK) return st;
      if ((st = set_global_field(s, offsetof(Global, status), 0)) != MW_OK) return st;
      continue;
    }
    if (g.status) return status_error(g);
    if ((st = set_global_field(s, offsetof(Global, any_rebuild), 0)) != MW_OK) return st;
    MW_CUDA(cudaStreamSynchronize(s->stream));
    s->forces_valid = false;  // atoms were re-sorted; stored forces no longer line up
    s->list_built = true;
    if (max_count_out) *max_count_out = g.max_count;
    return MW_OK;
  }
  return fail(MW_ENLIST_OVERFLOW, "neighbour list kept overflowing");
}

mw_status mw_get_neighbors(mw_system* s, int* counts, int* nbr, int width) {
  if (!s || !counts || !nbr || width < 1) return fail(MW_EINVAL, "bad arguments");
  if (!s->state_set || !s->list_built) return fail(MW_ESTATE, "no neighbour list built yet");
  int* dc;
  int* dn;
  mw_status st;
  if ((st = dalloc(s, &dc, s->N)) != MW_OK) return st;
  if ((st = dalloc(s, &dn, (size_t)s->N * width)) != MW_OK) {
    dfree(s, dc);
    return st;
  }
  k_gather_neighbors<<<div_up(s->N, kThreads), kThreads, 0, s->stream>>>(s->d, dc, dn, width);
  cudaError_t e = cudaGetLastError();
  if (e == cudaSuccess) e = cudaMemcpyAsync(counts, dc, sizeof(int) * s->N, cudaMemcpyDeviceToHost, s->stream);
  // copy only the filled prefix per atom would need a host loop; copy all and let the caller read counts
  std::vector<int> tmp;
  if (e == cudaSuccess) {
    tmp.resize((size_t)s->N * width);
    e = cudaMemcpyAsync(tmp.data(), dn, sizeof(int) * tmp.size(), cudaMemcpyDeviceToHost, s->stream);
  }
  if (e == cudaSuccess) e = cudaStreamSynchronize(s->stream);
  dfree(s, dc);
  dfree(s, dn);
  if (e != cudaSuccess) return fail(MW_ECUDA, "neighbour copy failed: %s", cudaGetErrorString(e));
  for (int u = 0; u < s->N; ++u) {
    const int m = std::min(counts[u], width);
    std::memcpy(nbr + (size_t)u * width, tmp.data() + (size_t)u * width, sizeof(int) * m);
  }
  return MW_OK;
}

mw_status mw_energy_forces(mw_system* s, double* f, double* energy, double* virial) {
  Range range_("mw_energy_forces");
  if (!s) return fail(MW_EINVAL, "system is NULL");
  mw_status st;
  if ((st = ensure_forces(s)) != MW_OK) return st;
  if (f) {
    k_gather_forces<<<div_up(s->N, kThreads), kThreads, 0, s->stream>>>(s->d, s->d.stage, nullptr);
    MW_CUDA(cudaGetLastError());
    MW_CUDA(cudaMemcpyAsync(f, s->d.stage, sizeof(double) * 3 * (size_t)s->N, cudaMemcpyDeviceToHost, s->stream));
  }
  if (energy || virial) {
    double* e = s->eout;
    double* w = s->eout + 3 * (size_t)s->nbox;
    k_energy_out<<<div_up(s->nbox, kThreads), kThreads, 0, s->stream>>>(s->d, e, w);
    MW_CUDA(cudaGetLastError());
    if (energy) MW_CUDA(cudaMemcpyAsync(energy, e, sizeof(double) * 3 * s->nbox, cudaMemcpyDeviceToHost, s->stream));
    if (virial) MW_CUDA(cudaMemcpyAsync(virial, w, sizeof(double) * 6 * s->nbox, cudaMemcpyDeviceToHost, s->stream));
  }
  MW_CUDA(cudaStreamSynchronize(s->stream));
  return MW_OK;
}

mw_status mw_energy_forces_dev(mw_system* s, const double* x_dev, float* f_dev, double* energy_dev,
                               double* virial_dev) {
  if (!s) return fail(MW_EINVAL, "system is NULL");
  if (x_dev) {
    if (!s->state_set) return do_set_state(s, x_dev, nullptr, true) == MW_OK ? mw_energy_forces_dev(s, nullptr, f_dev, energy_dev, virial_dev) : MW_ECUDA;
    mw_status st;
    if ((st = flush_pending(s)) != MW_OK) return st;
    k_load_positions<<<div_up(s->N, kThreads), kThreads, 0, s->stream>>>(s->d, x_dev, s->boxid);
    MW_CUDA(cudaGetLastError());
    if ((st = flag_all(s)) != MW_OK) return st;
    s->forces_valid = false;
  }
  mw_status st;
  if ((st = ensure_forces(s)) != MW_OK) return st;
  if (f_dev) k_gather_forces<<<div_up(s->N, kThreads), kThreads, 0, s->stream>>>(s->d, nullptr, f_dev);
  if (energy_dev || virial_dev)
    k_energy_out<<<div_up(s->nbox, kThreads), kThreads, 0, s->stream>>>(s->d, energy_dev, virial_dev);
  MW_CUDA(cudaGetLastError());
  MW_CUDA(cudaStreamSynchronize(s->stream));
  return MW_OK;
}

mw_status mw_forces_async(mw_system* s) {
  if (!s) return fail(MW_EINVAL, "system is NULL");
  mw_status st;
  if ((st = ensure_forces(s)) != MW_OK) return st;
  k_prep_force<<<div_up(std::max(s->N, s->nbox), kThreads), kThreads, 0, s->stream>>>(s->d, 1);
  launch_force(s);
  MW_CUDA(cudaGetLastError());
  return MW_OK;
}

mw_status mw_step(mw_system* s, const mw_integrator* integ, int nsteps, mw_thermo* last) {
  Range range_("mw_step");
  if (!s) return fail(MW_EINVAL, "system is NULL");
  if (nsteps < 0) return fail(MW_EINVAL, "nsteps < 0");
  mw_status st;
  if ((st = validate_integ(s, integ)) != MW_OK) return st;
  s->g_known_valid = false;  // set again only if ensure_forces reads the status block now
  if ((st = ensure_forces(s)) != MW_OK) return st;
  bool fetched = false;  // the run's last record came back with its final status read
  if (nsteps > 0) {
    int eng = s->engine;
    if (eng == MW_ENGINE_AUTO) eng = s->tuned_engine >= 0 ? s->tuned_engine : MW_ENGINE_PERSISTENT;
    if (eng == MW_ENGINE_PERSISTENT && !persistent_available(s)) eng = MW_ENGINE_GRAPH;
    s->engine_used = eng;
    st = eng == MW_ENGINE_PERSISTENT ? run_persistent_engine(s, nsteps, last, &fetched)
                                     : run_graph_engine(s, nsteps, last, &fetched, eng == MW_ENGINE_PLAIN);
    s->g_known_valid = false;
    if (st != MW_OK) {
      s->forces_valid = false;  // the state of an interrupted step is not a state to report forces of
      s->order_ok = false;
      return st;
    }
    s->list_built = true;
  }
  if (last && !fetched) return mw_get_thermo(s, last);
  return MW_OK;
}

mw_status mw_step_async(mw_system* s, const mw_integrator* integ, int nsteps) {
  Range range_("mw_step_async");
  if (!s) return fail(MW_EINVAL, "system is NULL");
  if (nsteps < 0) return fail(MW_EINVAL, "nsteps < 0");
  mw_status st;
  if ((st = validate_integ(s, integ)) != MW_OK) return st;
  if ((st = ensure_forces(s)) != MW_OK) return st;
  if (nsteps == 0) return MW_OK;
  int eng = s->engine;
  if (eng == MW_ENGINE_AUTO) eng = s->tuned_engine >= 0 ? s->tuned_engine : MW_ENGINE_PERSISTENT;
  if (eng == MW_ENGINE_PERSISTENT && !persistent_available(s)) eng = MW_ENGINE_GRAPH;
  s->engine_used = eng;
  if ((st = prime_thermostat(s)) != MW_OK) return st;
  s->record_pending = true;
  if (eng == MW_ENGINE_PERSISTENT) return enqueue_persistent(s, nsteps);
  if (eng == MW_ENGINE_PLAIN) return launch_plain_steps(s, nsteps);
  if (s->graph_dirty || !s->graph1) {
    if ((st = capture_graphs(s, 16)) != MW_OK) return st;
  }
  for (int k = 0; k < nsteps / s->graphK_steps; ++k) MW_CUDA(cudaGraphLaunch(s->graphK, s->stream));
  for (int k = 0; k < nsteps % s->graphK_steps; ++k) MW_CUDA(cudaGraphLaunch(s->graph1, s->stream));
  return MW_OK;
}

mw_status mw_sync(mw_system* s) {
  if (!s) return fail(MW_EINVAL, "system is NULL");
  Global g;
  mw_status st;
  if ((st = read_global(s, &g)) != MW_OK) return st;
  s->host_step = (long long)g.step;
  if (g.status == ST_GRID) {  // the run stopped at a step boundary: ready to continue
    if ((st = regrid(s)) != MW_OK) return st;
    s->graph_dirty = true;
  }
  if (g.status) s->order_ok = false;
  return status_error(g);
}

mw_status mw_get_thermo(mw_system* s, mw_thermo* out) {
  if (!s || !out) return fail(MW_EINVAL, "bad arguments");
  if (!s->state_set) return fail(MW_ESTATE, "no state set");
  mw_status st;
  if ((st = ensure_forces(s)) != MW_OK) return st;
  if ((st = enqueue_thermo(s)) != MW_OK) return st;
  MW_CUDA(cudaStreamSynchronize(s->stream));
  unpack_thermo(s, out);
  return MW_OK;
}

mw_status mw_get_box(mw_system* s, double* box) {
  if (!s || !box) return fail(MW_EINVAL, "bad arguments");
  mw_status st;
  if ((st = pull_boxes(s)) != MW_OK) return st;
  for (int b = 0; b < s->nbox; ++b)
    for (int k = 0; k < 3; ++k) box[3 * b + k] = s->boxes[b].L[k];
  return MW_OK;
}

mw_status mw_set_phase_marks(mw_system* s, int cap) {
  if (!s || cap < 0 || cap > (1 << 20)) return fail(MW_EINVAL, "cap must be in [0, 2^20]");
  mw_status st;
  if (cap > s->d.marks_cap) {
    dfree(s, s->d.marks);
    s->d.marks = nullptr;
    if ((st = dalloc(s, &s->d.marks, (size_t)cap * kPhaseMarks)) != MW_OK) return st;
  }
  if (cap == 0) {
    dfree(s, s->d.marks);
    s->d.marks = nullptr;
  }
  if (s->d.marks)
    MW_CUDA(cudaMemsetAsync(s->d.marks, 0, sizeof(unsigned long long) * (size_t)cap * kPhaseMarks, s->stream));
  s->d.marks_cap = cap;
  s->graph_dirty = true;
  return MW_OK;
}

mw_status mw_get_phase_marks(mw_system* s, unsigned long long* out, int cap) {
  if (!s || !out || cap < 0) return fail(MW_EINVAL, "bad arguments");
  if (cap > s->d.marks_cap) return fail(MW_EINVAL, "cap %d exceeds the %d steps recorded", cap, s->d.marks_cap);
  if (cap == 0) return MW_OK;
  MW_CUDA(cudaMemcpyAsync(out, s->d.marks, sizeof(unsigned long long) * (size_t)cap * kPhaseMarks,
                          cudaMemcpyDeviceToHost, s->stream));
  MW_CUDA(cudaStreamSynchronize(s->stream));
  return MW_OK;
}

mw_status mw_set_wait_limit(mw_system* s, double seconds) {
  if (!s || !(seconds >= 0.0) || !(seconds <= 60.0)) return fail(MW_EINVAL, "wait limit must be in [0, 60] s");
  s->wait_ns = (unsigned long long)(seconds * 1e9);
  return MW_OK;
}

mw_status mw_set_engine(mw_system* s, int engine) {
  if (!s || engine < MW_ENGINE_AUTO || engine > MW_ENGINE_PLAIN) return fail(MW_EINVAL, "bad engine");
  if (engine == MW_ENGINE_PLAIN && s->nsp > 1) return fail(MW_EINVAL, "the plain engine has one species only");
  s->engine = engine;
  return MW_OK;
}

mw_status mw_set_nbr_width(mw_system* s, int width) {
  if (!s || width < 1) return fail(MW_EINVAL, "bad width");
  mw_status st;
  if ((st = alloc_nbr(s, width)) != MW_OK) return st;
  // Forces at the current positions stay valid; the list is rebuilt in the
  // rebuild phase of the next step (or of the next force evaluation).
  if (s->state_set) {
    if ((st = flag_all(s)) != MW_OK) return st;
  }
  MW_CUDA(cudaStreamSynchronize(s->stream));
  return MW_OK;
}

mw_status mw_get_info(mw_system* s, mw_info* out) {
  if (!s || !out) return fail(MW_EINVAL, "bad arguments");
  Global g{};
  mw_status st;
  if ((st = read_global(s, &g)) != MW_OK) return st;
  out->nbox = s->nbox;
  out->n_total = s->N;
  out->nbr_width = s->W;
  out->max_count = g.max_count;
  out->ncell_total = s->ncell;
  out->engine = s->engine_used;
  out->persistent_blocks = s->pers_blocks;
  out->persistent_threads = kPersThreads;
  out->r_list = r_list(s);
  out->npairs = s->npairs;
  out->ntriplets = s->ntrip;
  out->rebuild_steps = g.rebuild_steps;
  out->regrids = s->regrids;
  out->species = s->nsp;
  out->species_moments = (s->nsp > 1 && s->sp_moment) ? 1 : 0;
  out->force_lanes = force_shape_lanes(s->force_shape);
  out->force_blocks_per_sm = force_shape_blocks(s->force_shape);
  out->force_owner = force_shape_owner(s->force_shape) ? 1 : 0;
  return MW_OK;
}

// Diagnostic switch (not in mw.h's stable set): count legs and triplets in
// the force kernel (atomics; slows it down).
mw_status mw_set_count_terms(mw_system* s, int on) {
  if (!s) return fail(MW_EINVAL, "system is NULL");
  s->count_terms = on ? 1 : 0;
  s->forces_valid = false;
  s->graph_dirty = true;
  mw_status st;
  if ((st = set_global_field(s, offsetof(Global, count_terms), s->count_terms)) != MW_OK) return st;
  MW_CUDA(cudaStreamSynchronize(s->stream));
  return MW_OK;
}

}  // extern "C"

// ===========================================================================
// Entry point for callers that cannot allocate device memory.
//
// Some callers of this library may not call cudaMalloc: code running inside a
// captured or externally managed memory pool, plugins whose host application
// owns all device allocations, or processes that have pinned their footprint
// up front.  mw_energy_forces_noalloc serves them: the caller passes device
// inputs and outputs, and every piece of scratch (fixed-point positions, cell
// lists, neighbour list, force accumulators, counters) lives in the one
// file-scope array below.  Each GPU that loads the library holds that array
// (MW_NOALLOC_SCRATCH_BYTES) until the process exits.
//
// In host code the symbol g_noalloc_scratch is only a host-side stand-in; its
// device address is fetched once per device with cudaGetSymbolAddress (on the
// first call made while that device is current) and cached.  Every call
// shares the array and leaves its contents behind: each call clears what must
// start at zero, and calls whose work overlaps on the GPU (different streams
// with no ordering between them) race on it.
// ===========================================================================

namespace {

constexpr size_t na_align(size_t x) { return (x + 255) / 256 * 256; }
constexpr size_t kNaQ = 0;                                                      // uint4 q[MAX]
constexpr size_t kNaTQ = kNaQ + na_align(sizeof(uint4) * MW_NOALLOC_MAX_ATOMS);  // uint4 tq[MAX]
constexpr size_t kNaF = kNaTQ + na_align(sizeof(uint4) * MW_NOALLOC_MAX_ATOMS);  // float4 f[MAX]
constexpr size_t kNaCell = kNaF + na_align(sizeof(float4) * MW_NOALLOC_MAX_ATOMS);
constexpr size_t kNaRank = kNaCell + na_align(sizeof(int) * MW_NOALLOC_MAX_ATOMS);
constexpr size_t kNaTid = kNaRank + na_align(sizeof(int) * MW_NOALLOC_MAX_ATOMS);
constexpr size_t kNaCnt = kNaTid + na_align(sizeof(int) * MW_NOALLOC_MAX_ATOMS);
constexpr size_t kNaOver = kNaCnt + na_align(sizeof(int) * MW_NOALLOC_MAX_ATOMS);
constexpr size_t kNaNbr = kNaOver + na_align(sizeof(int) * MW_NOALLOC_MAX_ATOMS);
constexpr size_t kNaCellCnt = kNaNbr + na_align(sizeof(int) * (size_t)MW_NOALLOC_MAX_ATOMS * MW_NOALLOC_MAX_WIDTH);
constexpr size_t kNaCellStart = kNaCellCnt + na_align(sizeof(int) * MW_NOALLOC_MAX_CELLS);
constexpr size_t kNaCellBox = kNaCellStart + na_align(sizeof(int) * (MW_NOALLOC_MAX_CELLS + 1));
constexpr size_t kNaBox = kNaCellBox + na_align(sizeof(int) * MW_NOALLOC_MAX_CELLS);
constexpr size_t kNaBst = kNaBox + na_align(sizeof(Box));
constexpr size_t kNaGlobal = kNaBst + na_align(sizeof(BoxState));
constexpr size_t kNaEnd = kNaGlobal + na_align(sizeof(Global));
static_assert(kNaEnd <= MW_NOALLOC_SCRATCH_BYTES, "no-alloc scratch layout exceeds its stated size");

__device__ __align__(256) unsigned char g_noalloc_scratch[MW_NOALLOC_SCRATCH_BYTES];

constexpr int kNaMaxDevices = 64;
// Device address of the array, per device; each slot is written once (by the
// first call that finds it empty; concurrent first calls store the same
// value).  A cudaDeviceReset between calls is not supported: the cached
// address would belong to the old context.
std::atomic<unsigned char*> g_na_base[kNaMaxDevices];

// Positions (AoS doubles, caller's order) -> fixed point, box 0.  The same
// conversion as the regular path (box fraction, its 64-bit fraction, then the
// 32-bit rounding), so both entry points see the same coordinates.  A
// non-finite value is replaced by 0 and reported (ST_INPUT, the atom in
// err_index); the host then refuses the call.
__global__ void k_na_load(Dev d, const double* __restrict__ x) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N) return;
  const Box& bx = d.box[0];
  unsigned long long p[3];
  for (int k = 0; k < 3; ++k) {
    double v = x[3 * (size_t)i + k];
    if (!isfinite(v)) {
      set_status(d.g, ST_INPUT);
      d.g->err_index = i;
      v = 0.0;
    }
    v /= bx.L[k];
    v -= floor(v);
    if (v >= 1.0) v -= 1.0;
    if (v < 0.0) v = 0.0;
    p[k] = frac64_of(v);
  }
  d.q[i] = make_uint4(q_of(p[0]), q_of(p[1]), q_of(p[2]), 0u);
}

// Cell-sorted copy of the fixed-point positions and their original indices.
__global__ void k_na_scatter(Dev d, uint4* __restrict__ tq) {
  const int i = blockIdx.x * blockDim.x + threadIdx.x;
  if (i >= d.N || d.g->status) return;
  const int p = d.cell_start[d.cell[i]] + d.rank[i];
  tq[p] = d.q[i];
  d.tid[p] = i;
}

// Sorted forces -> caller's order; energies and virial of the box.
// Nothing is written after a device error (the sorted order may then be
// incomplete, and the host reports the error instead).
__global__ void k_na_out(Dev d, float* __restrict__ f, double* __restrict__ e, double* __restrict__ w) {
  if (*(volatile int*)&d.g->status) return;
  const int p = blockIdx.x * blockDim.x + threadIdx.x;
  if (p < d.N && f) {
    const int u = d.tid[p];
    const float4 F = d.f[p];
    f[3 * (size_t)u] = F.x;
    f[3 * (size_t)u + 1] = F.y;
    f[3 * (size_t)u + 2] = F.z;
  }
  if (p == 0) {
    const double* ew = d.bst[0].ew[0];
    if (e) {
      e[0] = ew[0] + ew[1];
      e[1] = ew[0];
      e[2] = ew[1];
    }
    if (w)
      for (int k = 0; k < 6; ++k) w[k] = ew[2 + k];
  }
}

mw_status na_base(unsigned char** out) {
  int dev = 0;
  MW_CUDA(cudaGetDevice(&dev));
  if (dev < 0 || dev >= kNaMaxDevices) return fail(MW_EINVAL, "device index %d out of range", dev);
  unsigned char* b = g_na_base[dev].load(std::memory_order_acquire);
  if (!b) {
    void* p = nullptr;
    cudaError_t e = cudaGetSymbolAddress(&p, g_noalloc_scratch);
    if (e != cudaSuccess || !p) return fail(MW_ECUDA, "cudaGetSymbolAddress failed: %s", cudaGetErrorString(e));
    b = (unsigned char*)p;
    g_na_base[dev].store(b, std::memory_order_release);
  }
  *out = b;
  return MW_OK;
}

}  // namespace

extern "C" mw_status mw_energy_forces_noalloc(int n, const double box[3], const mw_params* prm, double skin,
                                              const double* x_dev, float* f_dev, double* energy_dev,
                                              double* virial_dev, void* stream) {
  if (n < 2 || !box || !x_dev) return fail(MW_EINVAL, "need n >= 2, box and x_dev");
  {
    // every call ends with a device-to-host read and a stream synchronisation,
    // which a capturing stream cannot do (and the capture would be invalidated)
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    MW_CUDA(cudaStreamIsCapturing((cudaStream_t)stream, &cs));
    if (cs != cudaStreamCaptureStatusNone)
      return fail(MW_EINVAL, "mw_energy_forces_noalloc cannot run on a stream that is being captured");
  }
  if (n > MW_NOALLOC_MAX_ATOMS)
    return fail(MW_EINVAL, "n = %d exceeds the no-alloc limit of %d atoms", n, MW_NOALLOC_MAX_ATOMS);
  mw_status st;
  if ((st = check_params(prm)) != MW_OK) return st;
  if (!(skin >= 0) || !std::isfinite(skin)) return fail(MW_EINVAL, "skin must be >= 0");
  const double rc = prm->a * prm->sigma, rl = rc + skin;
  Box bx;
  std::memset(&bx, 0, sizeof bx);
  long long ncell = 1;
  for (int k = 0; k < 3; ++k) {
    if (!(box[k] > 0) || !std::isfinite(box[k])) return fail(MW_EINVAL, "bad box edge");
    if (box[k] < 2.0 * rl) return fail(MW_EBOX, "box edge %d = %g A is shorter than 2 r_list = %g A", k, box[k], 2 * rl);
    bx.L[k] = box[k];
    bx.qs[k] = 4294967296.0 / box[k];
    bx.Lq[k] = (float)(box[k] / 4294967296.0);
    bx.nc[k] = std::max(1, (int)std::floor(box[k] / rl));
    ncell *= bx.nc[k];
  }
  if (ncell > MW_NOALLOC_MAX_CELLS)
    return fail(MW_EINVAL, "%lld cells exceed the no-alloc limit of %d (box too large)", ncell, MW_NOALLOC_MAX_CELLS);
  bx.lost = (float)(0.5 * std::min(box[0], std::min(box[1], box[2])));
  bx.off = 0;
  bx.n = n;
  bx.cell_off = 0;
  bx.volume = box[0] * box[1] * box[2];
  bx.Ndf = 3.0 * n - 3.0;
  bx.inv_ndf_kb = n > 1 ? 1.0 / (bx.Ndf * kKB) : 0.0;
  bx.p_fac = kATM / (3.0 * bx.volume);
  unsigned char* base = nullptr;
  if ((st = na_base(&base)) != MW_OK) return st;
  cudaStream_t sm = (cudaStream_t)stream;
  // this call's parameters and cleared counters
  mw_system tmp;  // host-side helper only (parameter packing); owns nothing on the device
  tmp.prm = *prm;
  tmp.skin = skin;
  make_fparams(&tmp);
  BoxState bs;
  std::memset(&bs, 0, sizeof bs);
  bs.s_endc = 1.0;
  bs.rebuild = 1;
  Global g{};
  g.any_rebuild = 1;
  MW_CUDA(cudaMemcpyAsync(base + kNaBox, &bx, sizeof bx, cudaMemcpyHostToDevice, sm));
  MW_CUDA(cudaMemcpyAsync(base + kNaBst, &bs, sizeof bs, cudaMemcpyHostToDevice, sm));
  MW_CUDA(cudaMemcpyAsync(base + kNaGlobal, &g, sizeof g, cudaMemcpyHostToDevice, sm));
  MW_CUDA(cudaMemsetAsync(base + kNaCellCnt, 0, sizeof(int) * (size_t)ncell, sm));
  MW_CUDA(cudaMemsetAsync(base + kNaCellBox, 0, sizeof(int) * (size_t)ncell, sm));
  Dev d{};
  d.N = n;
  d.W = MW_NOALLOC_MAX_WIDTH;
  d.ncell = (int)ncell;
  d.nbox = 1;
  d.q = (uint4*)(base + kNaQ);
  d.f = (float4*)(base + kNaF);
  d.cell = (int*)(base + kNaCell);
  d.rank = (int*)(base + kNaRank);
  d.tid = (int*)(base + kNaTid);
  d.nbr_cnt = (int*)(base + kNaCnt);
  d.over = (int*)(base + kNaOver);
  d.nbr = (int*)(base + kNaNbr);
  d.cell_cnt = (int*)(base + kNaCellCnt);
  d.cell_start = (int*)(base + kNaCellStart);
  d.cell_box = (int*)(base + kNaCellBox);
  d.box = (const Box*)(base + kNaBox);
  d.bst = (BoxState*)(base + kNaBst);
  d.g = (Global*)(base + kNaGlobal);
  uint4* tq = (uint4*)(base + kNaTQ);
  const int gb = div_up(n, kThreads);
  k_na_load<<<gb, kThreads, 0, sm>>>(d, x_dev);
  k_bin<<<gb, kThreads, 0, sm>>>(d);
  k_scan<<<1, kScanThreads, 0, sm>>>(d);
  k_na_scatter<<<gb, kThreads, 0, sm>>>(d, tq);
  Dev ds = d;  // the sorted view: neighbour list and forces work on the cell-sorted copy
  ds.q = tq;
  k_neigh<<<div_up(ncell * 32, kNeighThreads), kNeighThreads, 0, sm>>>(ds, tmp.fp.rl2);
  k_prep_force<<<gb, kThreads, 0, sm>>>(ds, 1);
  k_force<false><<<div_up(n, kFAtoms), kFThreads, 0, sm>>>(ds, tmp.fp);
  k_na_out<<<gb, kThreads, 0, sm>>>(ds, f_dev, energy_dev, virial_dev);
  MW_CUDA(cudaGetLastError());
  Global gout;
  MW_CUDA(cudaMemcpyAsync(&gout, base + kNaGlobal, sizeof gout, cudaMemcpyDeviceToHost, sm));
  MW_CUDA(cudaStreamSynchronize(sm));
  if (gout.status == ST_OVERFLOW)
    return fail(MW_ENLIST_OVERFLOW, "an atom has %d neighbours within r_list; the no-alloc limit is %d",
                gout.max_count, MW_NOALLOC_MAX_WIDTH);
  if (gout.status == ST_INPUT) return fail(MW_EINVAL, "non-finite position of atom %d", gout.err_index);
  if (gout.status) return status_error(gout);
  return MW_OK;
}
