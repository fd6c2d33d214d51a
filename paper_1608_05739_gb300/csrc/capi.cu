// capi.cu -- the extern "C" boundary declared in include/psatd.h: argument
// validation, plan ownership (scratch spectra and tables), the pass sequence
// of a PSATD step, FDTD dispatch, CUDA-event timing of every launch.
#include <cuda_runtime.h>
#include <stdint.h>

#include <cmath>
#include <cstdarg>
#include <cstdio>
#include <cstring>
#include <algorithm>
#include <mutex>
#include <string>
#include <type_traits>
#include <vector>

#include "../../include/psatd.h"
#include <nvtx3/nvToolsExt.h>

#include "farfield.h"
#include "launch.h"
#include "local.h"
#include "tables.h"

using namespace psatd;

namespace {

thread_local std::string g_err = "no error";

enum Slot { K_FWD_X = 0, K_FWD_Y = 1, K_PUSH = 2, K_INV_Y = 3, K_INV_X = 4, K_TABLES = 5, K_NSLOTS = 6 };
const char* kSlotNames[K_NSLOTS] = {"fwd_x_r2c", "fwd_y_c2c", "line_fft_push", "inv_y_c2c", "inv_x_c2r",
                                    "tables"};

struct EventPair {
  cudaEvent_t a, b;
};

// NVTX range for the profilers' timelines (a no-op unless a tool is attached):
// one per public step call and one per pass launch, named like the timing slots.
struct NvtxRange {
  explicit NvtxRange(const char* name) { nvtxRangePushA(name); }
  ~NvtxRange() { nvtxRangePop(); }
  NvtxRange(const NvtxRange&) = delete;
  NvtxRange& operator=(const NvtxRange&) = delete;
};

}  // namespace

struct psatd_plan_s {
  psatd_desc d;
  cudaStream_t st = nullptr;
  int device = 0;
  bool f32 = true;
  int ndim = 2, layout = 0, form = 0, n_in = 0, n_out = 0;
  int64_t nx = 0, ny = 0, nz = 1, nxh = 0, cs = 0;
  void* spec1 = nullptr;
  void* spec2 = nullptr;
  void* tw[3] = {nullptr, nullptr, nullptr};
  void* tab = nullptr;
  int64_t tab_e[3] = {1, 1, 1};
  size_t bytes = 0;
  bool coeffs_ready = false;
  double g0 = 0, r[3] = {1, 1, 1};
  std::string err = "no error";
  bool timing = false;
  std::vector<EventPair> ev[K_NSLOTS];
  std::vector<EventPair> pool;
  int npatch = 1;             // 2D batches: patches of this size class
  int64_t* d_off = nullptr;   // their element offsets in the caller's packed arrays (device)
  bool tc = false;            // tensor-core radix-16 stages (PSATD_MIXED_FP16 / _BF16)
  bool tc_bf16 = false;       // ... with split-BF16 operands (a third A piece)
  // launch configuration: lines per CTA of the passes fwd_x, fwd_y, inv_y, inv_x and of the
  // fused pass (-1: the built-in heuristic), and the fused pass's elements per thread
  // (8: radix-8 stages, 16: radix-16); set by psatd_plan_autotune
  int cfg_log_tb[4] = {-1, -1, -1, -1};
  int cfg_push_tb = -1;
  int push_ept = 8;
  int cfg_push_groups = -1;   // component groups of the fused pass (-1: the built-in choice)
  int maxsm = 0;              // opt-in shared memory per block of the plan's device
  int sm_bytes = 0;           // shared memory per SM of the plan's device
  int order = 0;                        // 0: nodes, exact k; p: staggered PSATD-p
  double* kp_d[3] = {nullptr, nullptr, nullptr};  // per axis k_p / g0 (n_i/2+1 entries)
  void* ph_d[3] = {nullptr, nullptr, nullptr};    // per axis half-cell phases (twiddle type)
  double* cw_d = nullptr;               // staggered Fornberg weights (p/2)
  void* gmat = nullptr;       // their split DFT matrices (kTcTail image, device)
  int* d_err = nullptr;       // device error word of the tensor-core passes
  int64_t caller_elems = 0;   // elements of each caller array (checked mode's extents)
};

namespace {

psatd_status fail(psatd_plan p, psatd_status s, const char* fmt, ...) {
  char buf[512];
  va_list ap;
  va_start(ap, fmt);
  vsnprintf(buf, sizeof buf, fmt, ap);
  va_end(ap);
  if (p) p->err = buf;
  else g_err = buf;
  return s;
}

psatd_status cuda_fail(psatd_plan p, cudaError_t e, const char* what) {
  return fail(p, PSATD_ERR_CUDA, "%s: %s", what, cudaGetErrorString(e));
}

bool pow2(int64_t v) { return v > 0 && (v & (v - 1)) == 0; }
// 3 * 2^k with k >= 4: the mixed-radix lengths of the FP32 passes (radix-3 first stage)
bool three_pow2(int64_t v) { return v >= 48 && v % 3 == 0 && pow2(v / 3); }
// 5 * 2^k with k >= 4: the radix-5 lengths of the FP32 passes
bool five_pow2(int64_t v) { return v >= 80 && v % 5 == 0 && pow2(v / 5); }
bool pos_finite(double v) { return std::isfinite(v) && v > 0; }

int layout_ndim(int layout) { return layout == PSATD_FIELDS_3D6 ? 3 : 2; }

// component slots of a layout / source form (see psatd_kernels.cuh)
void counts(int layout, int form, int* n_in, int* n_out) {
  const bool six = (layout == PSATD_FIELDS_3D6 || layout == PSATD_FIELDS_2D6);
  const int nf = six ? 6 : 3;
  const int nj = six ? 3 : (layout == PSATD_FIELDS_2D_TE ? 2 : 1);
  *n_out = nf;
  *n_in = nf + (form >= 1 ? nj : 0) + (form == 2 ? 2 : 0);
}

// which (E, B, J) components a layout uses
void present(int layout, bool e[3], bool b[3], bool j[3]) {
  for (int i = 0; i < 3; ++i) e[i] = b[i] = j[i] = true;
  if (layout == PSATD_FIELDS_2D_TE) {
    e[2] = b[0] = b[1] = j[2] = false;
  } else if (layout == PSATD_FIELDS_2D_TM) {
    e[0] = e[1] = b[2] = j[0] = j[1] = false;
  }
}

psatd_status validate_desc(psatd_plan p, const psatd_desc* d, bool psatd_limits) {
  if (!d) return fail(p, PSATD_ERR_INVALID_ARG, "desc is NULL");
  if (d->layout < 0 || d->layout > 3) return fail(p, PSATD_ERR_INVALID_ARG, "unknown layout %d", d->layout);
  if (d->ndim != layout_ndim(d->layout))
    return fail(p, PSATD_ERR_INVALID_ARG, "ndim %d does not match layout %d", d->ndim, d->layout);
  if ((d->flags & ~(psatd_limits ? (PSATD_FLAG_AUTOTUNE | PSATD_FLAG_PSTD | PSATD_FLAG_CHECKED |
                                     PSATD_FLAG_TEST_STALL_MMA | PSATD_FLAG_TEST_SHORT_EXTENT) : 0)) != 0)
    return fail(p, PSATD_ERR_INVALID_ARG, "unknown flags");
  if ((d->flags & PSATD_FLAG_TEST_SHORT_EXTENT) && !(d->flags & PSATD_FLAG_CHECKED))
    return fail(p, PSATD_ERR_INVALID_ARG, "PSATD_FLAG_TEST_SHORT_EXTENT needs PSATD_FLAG_CHECKED");
  if ((d->flags & PSATD_FLAG_TEST_STALL_MMA) && d->prec != PSATD_MIXED_FP16 && d->prec != PSATD_MIXED_BF16)
    return fail(p, PSATD_ERR_INVALID_ARG, "PSATD_FLAG_TEST_STALL_MMA applies to the mixed precisions only");
  if ((d->flags & PSATD_FLAG_PSTD) && d->src == PSATD_SRC_J_RHO)
    return fail(p, PSATD_ERR_INVALID_ARG, "PSTD takes J only (src must be NONE or J)");
  if (d->order != 0) {
    if (!psatd_limits)
      return fail(p, PSATD_ERR_INVALID_ARG, "order applies to the PSATD step only (the FDTD schemes are order 2)");
    if (d->order < 2 || d->order > 256 || (d->order & 1))
      return fail(p, PSATD_ERR_INVALID_ARG, "order must be 0 or an even number in [2, 256] (got %d)", d->order);
  }
  if (d->src < 0 || d->src > 2) return fail(p, PSATD_ERR_INVALID_ARG, "unknown source form %d", d->src);
  if (d->layout == PSATD_FIELDS_2D_TM && d->src == PSATD_SRC_J_RHO)
    return fail(p, PSATD_ERR_INVALID_ARG, "the TM layout has no rho-form (k.E = 0)");
  if (d->prec < 0 || d->prec > 3) return fail(p, PSATD_ERR_INVALID_ARG, "unknown precision %d", d->prec);
  if ((d->prec == PSATD_MIXED_FP16 || d->prec == PSATD_MIXED_BF16) && !psatd_limits)
    return fail(p, PSATD_ERR_UNSUPPORTED, "mixed precision applies to the PSATD step only");
  const int nd = d->ndim;
  for (int i = 0; i < nd; ++i)
    if (!pos_finite(d->d[i])) return fail(p, PSATD_ERR_INVALID_ARG, "d[%d] must be finite and > 0", i);
  if (!pos_finite(d->dt) || !pos_finite(d->c) || !pos_finite(d->eps0))
    return fail(p, PSATD_ERR_INVALID_ARG, "dt, c and eps0 must be finite and > 0");
  if (nd == 2 && d->n[2] != 1) return fail(p, PSATD_ERR_INVALID_ARG, "n[2] must be 1 in 2D");
  for (int i = 0; i < nd; ++i)
    if (d->n[i] < 2) return fail(p, PSATD_ERR_INVALID_ARG, "n[%d] = %lld too small", i, (long long)d->n[i]);
  if (psatd_limits) {
    // x is transformed as a complex line of nx/2 points, y and z as lines of n points:
    // powers of two, or (FP32 only) 3 * 2^k from 48 to 3072 or 5 * 2^k from 80 to 1280 points per line
    const bool mixed_ok = d->prec == PSATD_FP32;
    for (int i = 0; i < nd; ++i) {
      const int64_t L = i == 0 ? d->n[0] / 2 : d->n[i];
      const bool ok = (i > 0 || d->n[0] % 2 == 0) &&
                      ((pow2(L) && L >= 8 && d->n[i] <= 4096) || (mixed_ok && three_pow2(L) && d->n[i] <= 3072) ||
                       (mixed_ok && five_pow2(L) && L <= 1280));
      if (!ok) {
        const char* alt = !mixed_ok ? ""
                          : i == 0 ? ", 6 * 2^k in [96, 3072] or 10 * 2^k in [160, 2560]"
                                   : ", 3 * 2^k in [48, 3072] or 5 * 2^k in [80, 1280]";
        return fail(p, PSATD_ERR_UNSUPPORTED, "n[%d] must be a power of two in [%d, 4096]%s", i, i == 0 ? 16 : 8, alt);
      }
    }
  } else {
    for (int i = 0; i < nd; ++i)
      if (d->n[i] > (1LL << 20)) return fail(p, PSATD_ERR_UNSUPPORTED, "n[%d] too large", i);
  }
  return PSATD_OK;
}

bool aligned16(const void* q) { return (reinterpret_cast<uintptr_t>(q) & 15u) == 0; }

// A pointer the kernels may dereference on `device`: memory of that device,
// managed memory, or host memory allocated or registered through CUDA (pinned:
// under unified addressing the kernels use the host address itself, and the
// passes then read and write it over the host link).  Pageable host memory,
// and other devices' memory, are refused before any launch.
bool dev_accessible(const void* q, int device) {
  cudaPointerAttributes at;
  if (cudaPointerGetAttributes(&at, q) != cudaSuccess) {
    cudaGetLastError();
    return false;
  }
  if (at.type == cudaMemoryTypeDevice) return at.device == device;
  if (at.type == cudaMemoryTypeManaged) return true;
  if (at.type == cudaMemoryTypeHost) return at.devicePointer == q;
  return false;
}

// Collect the input slots of a step in kernel slot order; checks presence,
// absence and alignment of every pointer.
psatd_status gather_slots(psatd_plan p, const psatd_fields* f, const psatd_sources* s,
                          const void* in[kMaxComp], void* out[kMaxComp]) {
  if (!f) return fail(p, PSATD_ERR_INVALID_ARG, "fields is NULL");
  bool pe[3], pb[3], pj[3];
  present(p->layout, pe, pb, pj);
  const char* names = "xyz";
  for (int i = 0; i < 3; ++i) {
    if (pe[i] != (f->E[i] != nullptr))
      return fail(p, PSATD_ERR_INVALID_ARG, "E%c must be %s for this layout", names[i], pe[i] ? "non-NULL" : "NULL");
    if (pb[i] != (f->B[i] != nullptr))
      return fail(p, PSATD_ERR_INVALID_ARG, "B%c must be %s for this layout", names[i], pb[i] ? "non-NULL" : "NULL");
    if (f->E[i] && !aligned16(f->E[i])) return fail(p, PSATD_ERR_INVALID_ARG, "E%c not 16-byte aligned", names[i]);
    if (f->B[i] && !aligned16(f->B[i])) return fail(p, PSATD_ERR_INVALID_ARG, "B%c not 16-byte aligned", names[i]);
    if (f->E[i] && !dev_accessible(f->E[i], p->device))
      return fail(p, PSATD_ERR_INVALID_ARG, "E%c is not accessible from the plan's device", names[i]);
    if (f->B[i] && !dev_accessible(f->B[i], p->device))
      return fail(p, PSATD_ERR_INVALID_ARG, "B%c is not accessible from the plan's device", names[i]);
  }
  if (p->form != PSATD_SRC_NONE) {
    if (!s) return fail(p, PSATD_ERR_INVALID_ARG, "sources is NULL but the plan's source form needs them");
    for (int i = 0; i < 3; ++i) {
      if (pj[i] != (s->J[i] != nullptr))
        return fail(p, PSATD_ERR_INVALID_ARG, "J%c must be %s for this layout", names[i], pj[i] ? "non-NULL" : "NULL");
      if (s->J[i] && !aligned16(s->J[i])) return fail(p, PSATD_ERR_INVALID_ARG, "J%c not 16-byte aligned", names[i]);
      if (s->J[i] && !dev_accessible(s->J[i], p->device))
        return fail(p, PSATD_ERR_INVALID_ARG, "J%c is not accessible from the plan's device", names[i]);
    }
    if (p->form == PSATD_SRC_J_RHO) {
      if (!s->rho_n || !s->rho_np1) return fail(p, PSATD_ERR_INVALID_ARG, "rho-form needs rho_n and rho_np1");
      if (!aligned16(s->rho_n) || !aligned16(s->rho_np1))
        return fail(p, PSATD_ERR_INVALID_ARG, "rho arrays not 16-byte aligned");
      if (!dev_accessible(s->rho_n, p->device) || !dev_accessible(s->rho_np1, p->device))
        return fail(p, PSATD_ERR_INVALID_ARG, "rho arrays are not accessible from the plan's device");
    }
  }
  int k = 0;
  for (int i = 0; i < 3; ++i)
    if (pe[i]) { in[k] = f->E[i]; out[k] = f->E[i]; ++k; }
  for (int i = 0; i < 3; ++i)
    if (pb[i]) { in[k] = f->B[i]; out[k] = f->B[i]; ++k; }
  if (p->form >= 1)
    for (int i = 0; i < 3; ++i)
      if (pj[i]) { in[k] = s->J[i]; out[k] = nullptr; ++k; }
  if (p->form == 2) {
    in[k] = s->rho_n; out[k] = nullptr; ++k;
    in[k] = s->rho_np1; out[k] = nullptr; ++k;
  }
  return PSATD_OK;
}

void release(psatd_plan p) {
  void* bufs[] = {p->spec1, p->spec2, p->tw[0], p->tw[1], p->tw[2], p->tab, p->d_off, p->gmat, p->d_err,
                  p->kp_d[0], p->kp_d[1], p->kp_d[2], p->ph_d[0], p->ph_d[1], p->ph_d[2], p->cw_d};
  for (void* b : bufs)
    if (b) cudaFree(b);
  for (auto& v : p->ev) v.clear();
  for (auto& e : p->pool) {
    cudaEventDestroy(e.a);
    cudaEventDestroy(e.b);
  }
  p->pool.clear();
}

psatd_status alloc(psatd_plan p, void** ptr, size_t bytes, const char* what) {
  cudaError_t e = cudaMalloc(ptr, bytes);
  if (e != cudaSuccess) {
    *ptr = nullptr;
    cudaGetLastError();
    return fail(p, PSATD_ERR_OOM, "cudaMalloc of %zu bytes for %s failed: %s", bytes, what, cudaGetErrorString(e));
  }
  p->bytes += bytes;
  return PSATD_OK;
}

// threads per CTA a transposing pass may launch (the kernels' launch bounds)
int row_maxthr(int L, bool f32) { return row_ept(L) >= 20 || !f32 ? 256 : 512; }
// lines per CTA for a transposing pass of length L over `nb` lines (a divisor
// of nb; at most 16 lines: the row-dependent XOR of the transposed store
// spreads 16 lines over the banks, 32 would read one bank twice; the
// tensor-core variant goes to 32 where it needs that for 128 threads)
int pick_log_tb_raw(int L, int64_t nb, bool f32, bool tc) {
  const int T = L / row_ept(L);
  const int maxthr = row_maxthr(L, f32);
  int tb = 1;
  while (tb * 2 * T <= maxthr && tb * 2 <= 16 && nb % (tb * 2) == 0) tb *= 2;
  if (tc)
    while (tb * T < 128 && tb * 2 * T <= maxthr && tb * 2 <= 32 && nb % (tb * 2) == 0) tb *= 2;
  int lg = 0;
  while ((1 << lg) < tb) ++lg;
  return lg;
}
// lines per CTA of a forward transposing pass: as above; for the x rows (R2C,
// `rows`) at most 8 where a line's threads are whole warps (T a multiple of 32):
// the lines then synchronise only their own warps between stages (named barriers
// 1..8), measured faster than 16 lines on one CTA-wide barrier (1024^2 x: 23.0 ->
// 21.0 us).  The C2C y pass keeps 16 (its tile store writes 128-byte runs of z;
// 8 lines measured slower at 512 x 512 x 1024: 5.01 -> 5.42 ms).
int pick_log_tb(int L, int64_t nb, bool f32, bool tc = false, bool rows = false) {
  const int lg = pick_log_tb_raw(L, nb, f32, tc);
  const int T = L / row_ept(L);
  return (rows && !tc && T % 32 == 0 && lg > 3) ? 3 : lg;
}
// lines per CTA of an inverse transposing pass: half the forward rule's value
// before the cap above (the autotuner measured that faster at 2048^2 x, 1024^2 x,
// 256^3 x and y: the gathered bin pairs of fewer lines per CTA), keeping the
// tensor-core minimum
int pick_log_tb_inv(int L, int64_t nb, bool f32, bool tc = false) {
  const int lg = pick_log_tb_raw(L, nb, f32, tc);
  const int T = L / row_ept(L);
  if (lg == 0 || (tc && (T << (lg - 1)) < 128)) return lg;
  return lg - 1;
}

// shared memory of a transposing pass: one L-element buffer per line, or the
// [nk][tb + 1] transpose tile when the pass uses one (nk = 0: no tile)
size_t tpass_smem(int L, int log_tb, size_t nk, size_t csz) {
  const int tb = 1 << log_tb;
  const size_t a = (size_t)tb * L, b = nk * (size_t)(tb + 1);
  return (a > b ? a : b) * csz;
}

// lines per CTA of the fused last-axis pass: as few as make a whole warp (the
// autotuner found one line per CTA fastest at 256^3, 512^2 and 2048^2: the lines
// of a CTA only add barriers to each other); the tensor-core variant needs a
// multiple of 128 threads
int push_lines_per_cta(int L, int n_in, int64_t nlines, bool tc, bool f32, int ept) {
  (void)n_in;
  (void)nlines;
  (void)f32;
  const int T = L / ept;
  int tb = 1;
  while (tb * T < 32) tb *= 2;
  if (tc)
    while (tb * T < 128) tb *= 2;
  return tb;
}

// Component groups of the fused pass (psatd_kernels.cuh): 1, or 2 / 4 thread
// groups per line taking the components in turn, for FP32 plans without
// tensor-core stages whose lines have a multiple of 32 threads (named barriers
// per group: at most 15 per CTA; at most 512 threads; an even number of modes
// per thread in the push).
// Tensor-core plans take G = 2 only: component pairs in lockstep, one 128-row
// MMA group each (256 threads).
bool push_groups_ok(int L, int ept, int tb, int G, bool tc, bool f32) {
  if (G == 1) return true;
  if (L < ept) return false;
  const int T = L / ept;
  if (tc) return G == 2 && ept == 16 && T * tb == 128;
  if (!f32 || (G != 2 && G != 4)) return false;
  return T % 32 == 0 && (ept / G) % 2 == 0 && T * tb * G <= 512 && tb * G <= 15;
}
// shared memory of the fused pass: per line the n_in slots and one second
// exchange buffer per group (split-BF16's third A piece sits in a slot); the
// tensor-core pairs exchange in their own slots and keep the one spare buffer
// for the third A pieces
size_t push_smem(int n_in, int L, int tb, int G, size_t csz, bool tc = false) {
  return (size_t)tb * ((size_t)n_in + (size_t)(tc ? 1 : G)) * (size_t)L * csz;
}
// The built-in choice (measured on GB300 against the plain pass): two groups
// where lines have at least 64 threads and the plain pass keeps fewer than 12
// warps per SM resident for lack of shared memory (3D rho-form and 2D
// six-component J-form lines of 1024 points: 8 warps, 12 % faster with two
// groups); one group otherwise (the 2048^2 TE grid, 256^3, the 512-patch
// batch ran fastest with one).  sm_bytes: shared memory per SM.
int push_groups_default(int L, int ept, int tb, int n_in, bool tc, bool f32, size_t csz, int maxsm, int sm_bytes) {
  if (tc || !f32 || L < ept || sm_bytes <= 0) return 1;
  const int T = L / ept;
  if (T < 64) return 1;
  const size_t smem1 = push_smem(n_in, L, tb, 1, csz) + 1024;  // + the per-CTA reservation
  int ctas = (int)((size_t)sm_bytes / smem1);
  ctas = std::min(ctas, std::min(2048 / (T * tb), 32));
  if (ctas * T * tb / 32 >= 12) return 1;
  if (push_groups_ok(L, ept, tb, 2, tc, f32) && (maxsm <= 0 || push_smem(n_in, L, tb, 2, csz) <= (size_t)maxsm))
    return 2;
  return 1;
}

// split-BF16 passes: shared memory of the third A piece of `threads` threads
// (one 128-row piece per 128 threads), after the pass's exchange region
size_t tc_a3_bytes(psatd_plan p, int threads) {
  return p->tc_bf16 ? (size_t)(threads / 128) * TcGeom<16>::kAPiece : 0;
}

// Event pair around one launch on the plan's stream.  While the stream is being
// captured into a graph (multi-step batch calls) the events are captured as
// external event-record nodes, so that every replay records them again (a plain
// record during capture only expresses a dependency and is never timed).
struct TimedLaunch {
  psatd_plan p;
  int slot;
  cudaStream_t st;
  NvtxRange range;
  EventPair ep{};
  static void record(cudaEvent_t e, cudaStream_t st) {
    cudaStreamCaptureStatus cs = cudaStreamCaptureStatusNone;
    if (cudaStreamIsCapturing(st, &cs) == cudaSuccess && cs == cudaStreamCaptureStatusActive)
      cudaEventRecordWithFlags(e, st, cudaEventRecordExternal);
    else
      cudaEventRecord(e, st);
  }
  TimedLaunch(psatd_plan pl, int s) : TimedLaunch(pl, s, pl->st) {}
  TimedLaunch(psatd_plan pl, int s, cudaStream_t stream) : p(pl), slot(s), st(stream), range(kSlotNames[s]) {
    if (!p->timing) return;
    if (!p->pool.empty()) {
      ep = p->pool.back();
      p->pool.pop_back();
    } else {
      cudaEventCreate(&ep.a);
      cudaEventCreate(&ep.b);
    }
    record(ep.a, st);
  }
  ~TimedLaunch() {
    if (!p->timing) return;
    record(ep.b, st);
    p->ev[slot].push_back(ep);
  }
};

// Pass launchers by line length: powers of two, or the mixed lengths 3 * 2^k
// (float, no tensor-core stages; the size checks admit nothing else).
template <typename R, int TC>
cudaError_t fwd_T_any(int L, bool r2c, const PassGeom& g, cudaStream_t st, const LineIO& io, const void* tw,
                      int64_t in_sa0, int64_t in_sb, int64_t out_sa0, int64_t out_sk, const int64_t* a0_off = nullptr) {
  if (pow2(L)) return launch_fwd_T<R, TC>(L, r2c, g, st, io, tw, in_sa0, in_sb, out_sa0, out_sk, a0_off);
  if constexpr (std::is_same<R, float>::value && TC == 0) {
    if (three_pow2(L)) return launch_fwd_T3<R>(L, r2c, g, st, io, tw, in_sa0, in_sb, out_sa0, out_sk, a0_off);
    return launch_fwd_T5<R>(L, r2c, g, st, io, tw, in_sa0, in_sb, out_sa0, out_sk, a0_off);
  }
  return cudaErrorInvalidValue;
}
template <typename R, int TC>
cudaError_t inv_T_any(int L, bool c2r, const PassGeom& g, cudaStream_t st, const LineIO& io, const void* tw,
                      int64_t in_sa0, int64_t in_sk, int64_t out_sa0, int64_t out_sb, const int64_t* a0_off = nullptr) {
  if (pow2(L)) return launch_inv_T<R, TC>(L, c2r, g, st, io, tw, in_sa0, in_sk, out_sa0, out_sb, a0_off);
  if constexpr (std::is_same<R, float>::value && TC == 0) {
    if (three_pow2(L)) return launch_inv_T3<R>(L, c2r, g, st, io, tw, in_sa0, in_sk, out_sa0, out_sb, a0_off);
    return launch_inv_T5<R>(L, c2r, g, st, io, tw, in_sa0, in_sk, out_sa0, out_sb, a0_off);
  }
  return cudaErrorInvalidValue;
}

// Arguments of the fused pass of plan p over the spectra at sp (lines of Lline
// points, nlines of them).
template <typename R>
PushArgs<R> make_push_args(psatd_plan p, void* sp, int Lline, int64_t nlines) {
  PushArgs<R> a;
  std::memset(&a, 0, sizeof a);
  const bool chk = (p->d.flags & PSATD_FLAG_CHECKED) != 0;
  const int64_t shrink = (p->d.flags & PSATD_FLAG_TEST_SHORT_EXTENT) ? 1 : 0;
  a.spec = sp;
  a.cs = p->cs;
  a.tab = static_cast<const Coef<R>*>(p->tab);
  a.nlines = (int)nlines;
  a.n_in = p->n_in;
  a.n_out = p->n_out;
  a.form = p->form;
  a.ndim = p->ndim;
  a.nx_half = (int)(p->nx / 2);
  a.lines_per_patch = (int)p->nxh;
  a.ny = (int)p->ny;
  a.tab_row = Lline / 2 + 1;
  a.rx = (R)p->r[0];
  a.ry = (R)p->r[1];
  a.rz = (R)p->r[2];
  const double c = p->d.c, ic = 1.0 / c;
  a.c_h = (R)c;
  a.c_l = (R)(c - (double)a.c_h);
  a.ic_h = (R)ic;
  a.ic_l = (R)(ic - (double)a.ic_h);
  a.s_src = (R)(1.0 / (p->d.eps0 * c * p->g0));
  a.s_a6 = (R)(1.0 / (p->d.eps0 * c * c * p->g0));
  a.gmat = p->gmat;
  a.err = p->d_err;
  a.tc_ctl = (p->d.flags & PSATD_FLAG_TEST_STALL_MMA) ? kTcStallMma : 0;
  a.tab_ext = chk ? p->tab_e[0] * p->tab_e[1] * p->tab_e[2] - shrink : 0;
  a.chk_err = p->d_err;
  a.stag = p->order > 0 ? 1 : 0;
  a.scheme = (p->d.flags & PSATD_FLAG_PSTD) ? 1 : 0;
  a.p_h = (R)(0.5 * p->d.dt * p->g0);
  a.p_e = (R)(p->d.c * p->d.c * p->d.dt * p->g0);
  a.p_j = (R)(p->d.dt / p->d.eps0);
  a.inv_n = (R)(1.0 / ((double)p->nx * (double)p->ny * (double)p->nz));
  for (int i = 0; i < 3; ++i) {
    a.kp[i] = p->kp_d[i];
    a.ph[i] = p->ph_d[i];
  }
  return a;
}

template <typename R, int TC>
psatd_status run_step(psatd_plan p, const void* in[kMaxComp], void* out[kMaxComp]) {
  typedef typename Types<R>::C C;
  const size_t csz = sizeof(C);
  C* s1 = static_cast<C*>(p->spec1);
  C* s2 = static_cast<C*>(p->spec2);
  const int64_t nx = p->nx, ny = p->ny, nz = p->nz, nxh = p->nxh, cs = p->cs;
  const int Lx = (int)(nx / 2);
  cudaError_t e;
  LineIO io;
  std::memset(&io, 0, sizeof io);
  io.gmat = p->gmat;
  io.err = p->d_err;
  io.tc_ctl = (p->d.flags & PSATD_FLAG_TEST_STALL_MMA) ? kTcStallMma : 0;
  // checked mode: the extents every pass checks its index ranges against (the
  // test hook reports each array one element shorter than it is)
  const bool chk = (p->d.flags & PSATD_FLAG_CHECKED) != 0;
  const int64_t shrink = (p->d.flags & PSATD_FLAG_TEST_SHORT_EXTENT) ? 1 : 0;
  const int64_t ext_user = chk ? p->caller_elems - shrink : 0, ext_spec = chk ? cs - shrink : 0;
  io.chk_err = p->d_err;
  const size_t tail = TC ? (size_t)kTcTail : 0;  // tensor-core passes: matrices + mbarrier first

  // a0: z in 3D (strided), the patch in a 2D batch (offset table; spectra [c][patch][kx][y])
  const bool d3 = p->ndim == 3;
  const int64_t na0 = d3 ? nz : p->npatch;
  // pass 1: x rows (R2C), b = y -> spec1 [c][kx][z][y] (3D) / [c][patch][kx][y] (2D)
  {
    PassGeom g;
    g.log_tb = p->cfg_log_tb[0] >= 0 ? p->cfg_log_tb[0] : pick_log_tb(Lx, ny, p->f32, TC, true);
    g.grid = dim3((unsigned)(ny >> g.log_tb), (unsigned)na0, (unsigned)p->n_in);
    g.smem = tail + tpass_smem(Lx, g.log_tb, 0, csz) + tc_a3_bytes(p, (Lx / row_ept(Lx)) << g.log_tb);
    for (int c = 0; c < p->n_in; ++c) {
      io.in[c] = in[c];
      io.out[c] = s1 + c * cs;
    }
    io.in_ext = ext_user;
    io.out_ext = ext_spec;
    TimedLaunch tl(p, K_FWD_X);
    e = fwd_T_any<R, TC>(Lx, true, g, p->st, io, p->tw[0], d3 ? ny * nx : 0, nx, d3 ? ny : nxh * ny, nz * ny,
                        d3 ? nullptr : p->d_off);
    if (e != cudaSuccess) return cuda_fail(p, e, "fwd_x_r2c launch");
  }
  C* sp = s1;
  int Lline = (int)ny;
  int64_t nlines = nxh * p->npatch;
  if (p->ndim == 3) {
    // pass 2: y lines (C2C), b = z, a0 = kx: spec1 [c][kx][z][y] -> spec2 [c][kx][ky][z]
    PassGeom g;
    g.log_tb = p->cfg_log_tb[1] >= 0 ? p->cfg_log_tb[1] : pick_log_tb((int)ny, nz, p->f32, TC);
    g.grid = dim3((unsigned)(nz >> g.log_tb), (unsigned)nxh, (unsigned)p->n_in);
    g.smem = tail + tpass_smem((int)ny, g.log_tb, (size_t)ny, csz) +
             tc_a3_bytes(p, ((int)ny / row_ept((int)ny)) << g.log_tb);
    for (int c = 0; c < p->n_in; ++c) {
      io.in[c] = s1 + c * cs;
      io.out[c] = s2 + c * cs;
    }
    io.in_ext = ext_spec;
    io.out_ext = ext_spec;
    TimedLaunch tl(p, K_FWD_Y);
    e = fwd_T_any<R, TC>((int)ny, false, g, p->st, io, p->tw[1], nz * ny, ny, ny * nz, nz);
    if (e != cudaSuccess) return cuda_fail(p, e, "fwd_y_c2c launch");
    sp = s2;
    Lline = (int)nz;
    nlines = nxh * ny;
  }
  // fused last-axis pass
  {
    PushArgs<R> a = make_push_args<R>(p, sp, Lline, nlines);
    const void* twl = p->tw[p->ndim == 3 ? 2 : 1];
    {
      const int tb = p->cfg_push_tb > 0 ? p->cfg_push_tb
                                        : push_lines_per_cta(Lline, p->n_in, nlines, TC, p->f32, p->push_ept);
      int G = p->cfg_push_groups > 0
                  ? p->cfg_push_groups
                  : push_groups_default(Lline, p->push_ept, tb, p->n_in, TC, p->f32, csz, p->maxsm, p->sm_bytes);
      if (!push_groups_ok(Lline, p->push_ept, tb, G, TC, p->f32)) G = 1;
      const size_t smem = tail + push_smem(p->n_in, Lline, tb, G, csz, TC);
      const dim3 grid((unsigned)((nlines + tb - 1) / tb));
      TimedLaunch tl(p, K_PUSH);
      if (p->push_ept == 12 || p->push_ept == 20) {
        if constexpr (std::is_same<R, float>::value && TC == 0)
          e = p->push_ept == 12 ? launch_line_push3<R>(Lline, p->layout, grid, tb, G, smem, p->st, a, twl)
                                : launch_line_push5<R>(Lline, p->layout, grid, tb, G, smem, p->st, a, twl);
        else
          e = cudaErrorInvalidValue;
      } else if (p->push_ept == 16) {
        e = launch_line_push<R, TC, 16>(Lline, p->layout, grid, tb, G, smem, p->st, a, twl);
      } else {
        if constexpr (TC) e = cudaErrorInvalidValue;
        else e = launch_line_push<R, false, 8>(Lline, p->layout, grid, tb, G, smem, p->st, a, twl);
      }
      if (e != cudaSuccess) return cuda_fail(p, e, "line_fft_push launch");
    }
  }
  if (p->ndim == 3) {
    // pass 4: inverse y lines: spec2 [c][kx][ky][z] -> spec1 [c][kx][z][y]
    PassGeom g;
    g.log_tb = p->cfg_log_tb[2] >= 0 ? p->cfg_log_tb[2] : pick_log_tb_inv((int)ny, nz, p->f32, TC);
    g.grid = dim3((unsigned)(nz >> g.log_tb), (unsigned)nxh, (unsigned)p->n_out);
    g.smem = tail + tpass_smem((int)ny, g.log_tb, (size_t)ny, csz) +
             tc_a3_bytes(p, ((int)ny / row_ept((int)ny)) << g.log_tb);
    for (int c = 0; c < p->n_out; ++c) {
      io.in[c] = s2 + c * cs;
      io.out[c] = s1 + c * cs;
    }
    io.in_ext = ext_spec;
    io.out_ext = ext_spec;
    TimedLaunch tl(p, K_INV_Y);
    e = inv_T_any<R, TC>((int)ny, false, g, p->st, io, p->tw[1], ny * nz, nz, nz * ny, ny);
    if (e != cudaSuccess) return cuda_fail(p, e, "inv_y_c2c launch");
  }
  // last pass: inverse x rows (C2R): spec1 -> out [z][y][x] (3D) / packed patches (2D)
  {
    PassGeom g;
    g.log_tb = p->cfg_log_tb[3] >= 0 ? p->cfg_log_tb[3] : pick_log_tb_inv(Lx, ny, p->f32, TC);
    g.grid = dim3((unsigned)(ny >> g.log_tb), (unsigned)na0, (unsigned)p->n_out);
    g.smem = tail + tpass_smem(Lx, g.log_tb, 0, csz) + tc_a3_bytes(p, (Lx / row_ept(Lx)) << g.log_tb);
    for (int c = 0; c < p->n_out; ++c) {
      io.in[c] = s1 + c * cs;
      io.out[c] = out[c];
    }
    io.in_ext = ext_spec;
    io.out_ext = ext_user;
    TimedLaunch tl(p, K_INV_X);
    e = inv_T_any<R, TC>(Lx, true, g, p->st, io, p->tw[0], d3 ? ny : nxh * ny, nz * ny, d3 ? ny * nx : 0, nx,
                        d3 ? nullptr : p->d_off);
    if (e != cudaSuccess) return cuda_fail(p, e, "inv_x_c2r launch");
  }
  return PSATD_OK;
}

psatd_status step_once(psatd_plan p, const void* in[kMaxComp], void* out[kMaxComp]) {
  psatd_status s;
  if (p->tc) s = p->tc_bf16 ? run_step<float, 2>(p, in, out) : run_step<float, 1>(p, in, out);
  else s = p->f32 ? run_step<float, 0>(p, in, out) : run_step<double, 0>(p, in, out);
  if (s == PSATD_OK && (p->d.flags & PSATD_FLAG_CHECKED)) {
    cudaError_t e = launch_nonfinite(p->f32, out, p->n_out, p->d_off, p->npatch, p->nx * p->ny * p->nz, p->d_err,
                                     p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "non-finite scan launch");
  }
  return s;
}

// Shape checks of the tensor-core variant: every transposing pass and the fused
// pass run with a multiple of 128 threads per CTA (one MMA row per thread).
psatd_status check_tc_shape(psatd_plan p, int maxsm) {
  const int Lx = (int)(p->nx / 2);
  const int Ll = (int)(p->ndim == 3 ? p->nz : p->ny);
  if (Lx < 16 || Ll < 16 || (p->ndim == 3 && p->ny < 16))
    return fail(nullptr, PSATD_ERR_UNSUPPORTED, "mixed precision needs nx >= 32 and ny, nz >= 16");
  struct { int L; int64_t nb; } rows[2] = {{Lx, p->ny}, {(int)p->ny, p->nz}};
  for (int i = 0; i < (p->ndim == 3 ? 2 : 1); ++i) {
    const int T = rows[i].L / row_ept(rows[i].L);
    if ((T << pick_log_tb(rows[i].L, rows[i].nb, true, true)) < 128)
      return fail(nullptr, PSATD_ERR_UNSUPPORTED,
                  "mixed precision: a line pass of length %d over %lld lines has fewer than 128 threads per CTA",
                  rows[i].L, (long long)rows[i].nb);
  }
  const int64_t nlines = p->ndim == 3 ? p->nxh * p->ny : p->nxh * p->npatch;
  const int tb = push_lines_per_cta(Ll, p->n_in, nlines, true, true, 16);
  const size_t smem = (size_t)kTcTail + push_smem(p->n_in, Ll, tb, 1, 8);
  if (maxsm > 0 && smem > (size_t)maxsm)
    return fail(nullptr, PSATD_ERR_UNSUPPORTED, "mixed precision: last-axis length %d needs %zu bytes of shared memory",
                Ll, smem);
  return PSATD_OK;
}

// ---------------------------------------------------------------- autotuner
// Knobs: lines per CTA of each transposing pass (fwd_x, fwd_y, inv_y, inv_x)
// and, for the fused pass, its radix schedule (8 or 16 elements per thread:
// radix-8 or radix-16 stages) with its lines per CTA.  Every valid candidate
// of every knob is timed on the plan's stream (CUDA events around each launch)
// over `reps` steps on zero-filled scratch fields; the passes are independent,
// so round i sets every knob to its i-th candidate and one series of steps
// times them all.  Results are cached per (precision, layout, source form,
// sizes, patch count) for the process.
struct TuneCfg {
  int log_tb[4];
  int push_tb, push_ept;
  int push_groups = -1;
};
struct TuneKey {
  int prec, layout, form, npatch, order, flags;
  int64_t n[3];
  bool operator==(const TuneKey& o) const {
    return prec == o.prec && layout == o.layout && form == o.form && npatch == o.npatch && order == o.order &&
           flags == o.flags &&
           n[0] == o.n[0] &&
           n[1] == o.n[1] && n[2] == o.n[2];
  }
};
std::mutex g_tune_mutex;
std::vector<std::pair<TuneKey, TuneCfg>> g_tune_cache;

TuneKey tune_key(psatd_plan p) {
  return TuneKey{p->d.prec, p->layout, p->form, p->npatch, p->order, p->d.flags & PSATD_FLAG_PSTD,
                 {p->nx, p->ny, p->nz}};
}
void apply_cfg(psatd_plan p, const TuneCfg& c) {
  for (int i = 0; i < 4; ++i) p->cfg_log_tb[i] = c.log_tb[i];
  p->cfg_push_tb = c.push_tb;
  p->push_ept = c.push_ept;
  p->cfg_push_groups = c.push_groups;
}

psatd_status regen_push_twiddles(psatd_plan p) {
  if (p->ndim < 2) return PSATD_OK;
  const int i = p->ndim - 1;
  const int L = (int)(i == 2 ? p->nz : p->ny);
  cudaError_t e = launch_twiddles(p->tw[i], L, p->push_ept, false, p->f32, p->st);
  return e == cudaSuccess ? PSATD_OK : cuda_fail(p, e, "twiddle table launch");
}

// Valid launch shapes of every knob: rows[k] = log2(lines per CTA) of
// transposing pass k (empty if the pass does not exist), push = (elements per
// thread, lines per CTA, component groups) of the fused pass.
struct PushShape {
  int ept, tb, groups;
};
struct TuneSpace {
  std::vector<int> rows[4];
  std::vector<PushShape> push;
  int rowL[4];
  int Ll;
};

TuneSpace tune_space(psatd_plan p) {
  TuneSpace ts;
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
  const size_t csz = p->f32 ? 8 : 16;
  const size_t tail = p->tc ? (size_t)kTcTail : 0;
  const int Lx = (int)(p->nx / 2);
  ts.Ll = (int)(p->ndim == 3 ? p->nz : p->ny);
  const int64_t nlines = p->ndim == 3 ? p->nxh * p->ny : p->nxh * p->npatch;
  const int rowL[4] = {Lx, (int)p->ny, (int)p->ny, Lx};
  const int64_t rowNb[4] = {p->ny, p->nz, p->nz, p->ny};
  const size_t rowNk[4] = {0, (size_t)p->ny, (size_t)p->ny, 0};
  const bool rowOn[4] = {true, p->ndim == 3, p->ndim == 3, true};
  for (int k = 0; k < 4; ++k) {
    ts.rowL[k] = rowL[k];
    if (!rowOn[k]) continue;
    const int T = rowL[k] / row_ept(rowL[k]);
    const int maxthr = row_maxthr(rowL[k], p->f32);
    for (int lg = 0; (1 << lg) <= 32 && rowNb[k] % (1 << lg) == 0 && (T << lg) <= maxthr; ++lg) {
      if (p->tc && (T << lg) < 128) continue;
      if (maxsm > 0 && tail + tpass_smem(rowL[k], lg, rowNk[k], csz) + tc_a3_bytes(p, T << lg) > (size_t)maxsm)
        continue;
      ts.rows[k].push_back(lg);
    }
  }
  for (int ept : {8, 16, 12, 20}) {
    // powers of two: radix-8 or radix-16 stages (tensor cores: 16); 3 * 2^k: 12; 5 * 2^k: 20
    const bool allowed = pow2(ts.Ll) ? (ept == 8 || ept == 16) && (!p->tc || ept == 16) : ept == push_ept(ts.Ll);
    if (!allowed || ts.Ll < ept) continue;
    const int T = ts.Ll / ept;
    for (int tb = 1; tb * T <= (T > 256 ? T : 256); tb *= 2) {
      if (p->tc && (tb * T) % 128 != 0) continue;
      if (tb > 1 && tb / 2 >= nlines) break;
      for (int G : {1, 2, 4}) {
        if (!push_groups_ok(ts.Ll, ept, tb, G, p->tc, p->f32)) continue;
        if (maxsm > 0 && tail + push_smem(p->n_in, ts.Ll, tb, G, csz, p->tc) > (size_t)maxsm) continue;
        ts.push.push_back({ept, tb, G});
      }
    }
  }
  return ts;
}

psatd_status autotune(psatd_plan p, int reps, std::string* report) {
  if (reps < 1) reps = 1;
  const size_t rsz = p->f32 ? 4 : 8;
  TuneSpace ts = tune_space(p);
  std::vector<int>* rows = ts.rows;
  std::vector<PushShape>& push = ts.push;
  const int* rowL = ts.rowL;
  const int Ll = ts.Ll;
  const bool rowOn[4] = {true, p->ndim == 3, p->ndim == 3, true};
  for (int k = 0; k < 4; ++k)
    if (rowOn[k] && rows[k].empty())
      return fail(p, PSATD_ERR_UNSUPPORTED, "autotune: no valid launch shape for pass %d", k);
  if (push.empty()) return fail(p, PSATD_ERR_UNSUPPORTED, "autotune: no valid launch shape for the fused pass");
  // scratch fields (zero) and, for a batch class, contiguous patch offsets
  const size_t cells = (size_t)p->nx * p->ny * p->nz * p->npatch;
  void* fbuf = nullptr;
  cudaError_t e = cudaMalloc(&fbuf, (size_t)p->n_in * cells * rsz);
  if (e != cudaSuccess) {
    cudaGetLastError();
    return fail(p, PSATD_ERR_OOM, "autotune: scratch fields of %zu bytes", (size_t)p->n_in * cells * rsz);
  }
  int64_t* d_off2 = nullptr;
  int64_t* saved_off = p->d_off;
  psatd_status st = PSATD_OK;
  if (p->d_off) {
    std::vector<int64_t> offs(p->npatch);
    for (int i = 0; i < p->npatch; ++i) offs[i] = (int64_t)i * p->nx * p->ny;
    e = cudaMalloc(&d_off2, offs.size() * sizeof(int64_t));
    if (e == cudaSuccess) e = cudaMemcpy(d_off2, offs.data(), offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
    if (e != cudaSuccess) st = cuda_fail(p, e, "autotune: offset table");
    else p->d_off = d_off2;
  }
  if (st == PSATD_OK) {
    e = cudaMemsetAsync(fbuf, 0, (size_t)p->n_in * cells * rsz, p->st);
    if (e != cudaSuccess) st = cuda_fail(p, e, "autotune: clear");
  }
  const void* in[kMaxComp] = {};
  void* out[kMaxComp] = {};
  for (int c = 0; c < p->n_in; ++c) {
    in[c] = static_cast<char*>(fbuf) + c * cells * rsz;
    if (c < p->n_out) out[c] = const_cast<void*>(in[c]);
  }
  size_t rounds = push.size();
  for (int k = 0; k < 4; ++k) rounds = std::max(rounds, rows[k].size());
  std::vector<double> trow[4], tpush(push.size(), 1e30);
  for (int k = 0; k < 4; ++k) trow[k].assign(rows[k].size(), 1e30);
  const int slot_of[4] = {K_FWD_X, K_FWD_Y, K_INV_Y, K_INV_X};
  const bool was_timing = p->timing;
  const int saved_ept = p->push_ept;
  for (size_t r = 0; r < rounds && st == PSATD_OK; ++r) {
    for (int k = 0; k < 4; ++k)
      if (!rows[k].empty()) p->cfg_log_tb[k] = rows[k][std::min(r, rows[k].size() - 1)];
    const PushShape pc = push[std::min(r, push.size() - 1)];
    if (pc.ept != p->push_ept) {
      p->push_ept = pc.ept;
      if ((st = regen_push_twiddles(p)) != PSATD_OK) break;
    }
    p->cfg_push_tb = pc.tb;
    p->cfg_push_groups = pc.groups;
    if ((st = step_once(p, in, out)) != PSATD_OK) break;  // warm-up
    cudaStreamSynchronize(p->st);
    for (auto& v : p->ev) {
      for (auto& ev : v) p->pool.push_back(ev);
      v.clear();
    }
    p->timing = true;
    for (int i = 0; i < reps && st == PSATD_OK; ++i) st = step_once(p, in, out);
    p->timing = false;
    e = cudaStreamSynchronize(p->st);
    if (e != cudaSuccess && st == PSATD_OK) st = cuda_fail(p, e, "autotune: synchronise");
    auto avg = [&](int slot) {
      double ms = 0;
      for (auto& ev : p->ev[slot]) {
        float t = 0;
        if (cudaEventElapsedTime(&t, ev.a, ev.b) == cudaSuccess) ms += t;
      }
      return p->ev[slot].empty() ? 1e30 : ms / p->ev[slot].size();
    };
    for (int k = 0; k < 4; ++k)
      if (r < rows[k].size()) trow[k][r] = avg(slot_of[k]);
    if (r < push.size()) tpush[r] = avg(K_PUSH);
    for (auto& v : p->ev) {
      for (auto& ev : v) p->pool.push_back(ev);
      v.clear();
    }
  }
  p->timing = was_timing;
  p->d_off = saved_off;
  cudaStreamSynchronize(p->st);
  cudaFree(fbuf);
  if (d_off2) cudaFree(d_off2);
  if (st != PSATD_OK) {
    for (int k = 0; k < 4; ++k) p->cfg_log_tb[k] = -1;
    p->cfg_push_tb = -1;
    p->cfg_push_groups = -1;
    if (p->push_ept != saved_ept) {
      p->push_ept = saved_ept;
      regen_push_twiddles(p);
    }
    return st;
  }
  TuneCfg best{{-1, -1, -1, -1}, -1, p->push_ept};
  const char* names[4] = {"fwd_x", "fwd_y", "inv_y", "inv_x"};
  char buf[160];
  for (int k = 0; k < 4; ++k) {
    if (rows[k].empty()) continue;
    size_t b = std::min_element(trow[k].begin(), trow[k].end()) - trow[k].begin();
    best.log_tb[k] = rows[k][b];
    if (report) {
      std::snprintf(buf, sizeof buf, "%s L=%d:", names[k], rowL[k]);
      *report += buf;
      for (size_t i = 0; i < rows[k].size(); ++i) {
        std::snprintf(buf, sizeof buf, " tb=%d %.4fms%s", 1 << rows[k][i], trow[k][i], i == b ? "*" : "");
        *report += buf;
      }
      *report += "; ";
    }
  }
  size_t b = std::min_element(tpush.begin(), tpush.end()) - tpush.begin();
  best.push_ept = push[b].ept;
  best.push_tb = push[b].tb;
  best.push_groups = push[b].groups;
  if (report) {
    std::snprintf(buf, sizeof buf, "push L=%d:", Ll);
    *report += buf;
    for (size_t i = 0; i < push.size(); ++i) {
      std::snprintf(buf, sizeof buf, " radix%d tb=%d g=%d %.4fms%s", push[i].ept, push[i].tb, push[i].groups,
                    tpush[i], i == b ? "*" : "");
      *report += buf;
    }
  }
  apply_cfg(p, best);
  if ((st = regen_push_twiddles(p)) != PSATD_OK) return st;
  std::lock_guard<std::mutex> lock(g_tune_mutex);
  const TuneKey key = tune_key(p);
  for (auto& kv : g_tune_cache)
    if (kv.first == key) {
      kv.second = best;
      return PSATD_OK;
    }
  g_tune_cache.push_back({key, best});
  return PSATD_OK;
}

}  // namespace

extern "C" {

int32_t psatd_abi_version(void) { return PSATD_ABI_VERSION; }

static psatd_status plan_create_n(const psatd_desc* desc, void* cuda_stream, int npatch, psatd_plan* out) {
  *out = nullptr;
  psatd_status s = validate_desc(nullptr, desc, true);
  if (s != PSATD_OK) return s;
  psatd_plan p = new (std::nothrow) psatd_plan_s();
  if (!p) return fail(nullptr, PSATD_ERR_OOM, "host allocation failed");
  p->d = *desc;
  p->st = static_cast<cudaStream_t>(cuda_stream);
  p->f32 = desc->prec != PSATD_FP64;
  p->tc = desc->prec == PSATD_MIXED_FP16 || desc->prec == PSATD_MIXED_BF16;
  p->tc_bf16 = desc->prec == PSATD_MIXED_BF16;
  p->push_ept = push_ept((int)(desc->ndim == 3 ? desc->n[2] : desc->n[1]), p->tc);
  p->order = desc->order;
  p->ndim = desc->ndim;
  p->layout = desc->layout;
  p->form = desc->src;
  counts(p->layout, p->form, &p->n_in, &p->n_out);
  p->nx = desc->n[0];
  p->ny = desc->n[1];
  p->nz = p->ndim == 3 ? desc->n[2] : 1;
  p->nxh = p->nx / 2 + 1;
  p->npatch = npatch;
  p->cs = p->nxh * p->ny * p->nz * npatch;
  p->caller_elems = p->nx * p->ny * p->nz * npatch;  // batches and local decompositions set their packed size
  cudaGetDevice(&p->device);
  // push pass shared memory (one line per CTA at least)
  {
    const int L = (int)(p->ndim == 3 ? p->nz : p->ny);
    const size_t csz = p->f32 ? 8 : 16;
    const size_t need = push_smem(p->n_in, L, 1, 1, csz);
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
    p->maxsm = maxsm;
    cudaDeviceGetAttribute(&p->sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, p->device);
    if (maxsm > 0 && need > (size_t)maxsm) {
      psatd_status r = fail(nullptr, PSATD_ERR_UNSUPPORTED,
                            "last-axis length %d with %d components needs %zu bytes of shared memory (> %d)", L,
                            p->n_in, need, maxsm);
      delete p;
      return r;
    }
    if (p->tc) {
      psatd_status r = check_tc_shape(p, maxsm);
      if (r != PSATD_OK) {
        delete p;
        return r;
      }
    }
  }
  // wavenumber scale: k_i = g0 r_i m_i; FP32 plans use the float-rounded ratios
  p->g0 = 2.0 * M_PI / ((double)p->nx * desc->d[0]);
  const int64_t ns[3] = {p->nx, p->ny, p->nz};
  for (int i = 0; i < 3; ++i) {
    if (i >= p->ndim) {
      p->r[i] = 0.0;
      continue;
    }
    const double gi = 2.0 * M_PI / ((double)ns[i] * desc->d[i]);
    double ri = gi / p->g0;
    if (p->f32) ri = (double)(float)ri;
    p->r[i] = ri;
  }
  const size_t csz = p->f32 ? 8 : 16;
  const size_t spec_bytes = (size_t)p->n_in * (size_t)p->cs * csz;
  psatd_status a = alloc(p, &p->spec1, spec_bytes, "spectra");
  if (a == PSATD_OK && p->ndim == 3) a = alloc(p, &p->spec2, spec_bytes, "spectra (2)");
  const size_t wsz = p->f32 ? 16 : 16;
  for (int i = 0; i < p->ndim && a == PSATD_OK; ++i) a = alloc(p, &p->tw[i], (size_t)ns[i] * wsz, "twiddles");
  p->tab_e[0] = p->nx / 2 + 1;
  p->tab_e[1] = p->ny / 2 + 1;
  p->tab_e[2] = p->ndim == 3 ? p->nz / 2 + 1 : 1;
  const size_t ent = (size_t)p->tab_e[0] * p->tab_e[1] * p->tab_e[2];
  if (a == PSATD_OK) a = alloc(p, &p->tab, ent * (p->f32 ? sizeof(Coef<float>) : sizeof(Coef<double>)), "coefficients");
  if (a == PSATD_OK && p->tc) a = alloc(p, &p->gmat, 2 * TcGeom<16>::kGDir, "tensor-core DFT matrices");
  for (int i = 0; i < p->ndim && a == PSATD_OK && p->order > 0; ++i) {
    a = alloc(p, reinterpret_cast<void**>(&p->kp_d[i]), (size_t)(ns[i] / 2 + 1) * sizeof(double), "k_p table");
    if (a == PSATD_OK) a = alloc(p, &p->ph_d[i], (size_t)(ns[i] / 2 + 1) * 16, "staggering phases");
  }
  if (a == PSATD_OK && p->order > 0)
    a = alloc(p, reinterpret_cast<void**>(&p->cw_d), (size_t)(p->order / 2) * sizeof(double), "stencil weights");
  // the device error word (expired bounded waits, checked mode)
  if (a == PSATD_OK) a = alloc(p, reinterpret_cast<void**>(&p->d_err), sizeof(int), "error word");
  if (a == PSATD_OK) {
    cudaError_t e = cudaMemset(p->d_err, 0, sizeof(int));
    if (e != cudaSuccess) a = cuda_fail(p, e, "error word clear");
  }
  if (a != PSATD_OK) {
    g_err = p->err;
    release(p);
    delete p;
    return a;
  }
  *out = p;
  return PSATD_OK;
}

psatd_status psatd_plan_create(const psatd_desc* desc, void* cuda_stream, psatd_plan* out) {
  if (!out) return fail(nullptr, PSATD_ERR_INVALID_ARG, "out is NULL");
  return plan_create_n(desc, cuda_stream, 1, out);
}

psatd_status psatd_coeffs_init(psatd_plan p) {
  if (!p) return fail(nullptr, PSATD_ERR_INVALID_ARG, "plan is NULL");
  cudaError_t e;
  const int64_t ns[3] = {p->nx, p->ny, p->nz};
  {
    TimedLaunch tl(p, K_TABLES);
    for (int i = 0; i < p->ndim; ++i) {
      const int L = i == 0 ? (int)(ns[0] / 2) : (int)ns[i];
      const bool push_axis = (i == p->ndim - 1) && i > 0;
      e = launch_twiddles(p->tw[i], L, push_axis ? p->push_ept : row_ept(L), i == 0, p->f32, p->st);
      if (e != cudaSuccess) return cuda_fail(p, e, "twiddle table launch");
    }
    if (p->tc) {
      e = launch_tc_dftmat(p->gmat, p->tc_bf16, p->st);
      if (e != cudaSuccess) return cuda_fail(p, e, "tensor-core DFT matrix launch");
    }
    if (p->order > 0) {
      std::vector<double> C(p->order / 2);
      staggered_weights(p->order, C.data());
      e = cudaMemcpyAsync(p->cw_d, C.data(), C.size() * sizeof(double), cudaMemcpyHostToDevice, p->st);
      if (e != cudaSuccess) return cuda_fail(p, e, "stencil weight upload");
      for (int i = 0; i < p->ndim; ++i) {
        e = launch_kp_tables(p->kp_d[i], p->ph_d[i], p->cw_d, p->order / 2, (int)ns[i], p->d.d[i], p->g0, p->f32,
                             p->st);
        if (e != cudaSuccess) return cuda_fail(p, e, "k_p table launch");
      }
      e = cudaStreamSynchronize(p->st);  // the host weights are read by the copy above
      if (e != cudaSuccess) return cuda_fail(p, e, "stencil weight upload");
    }
    const double N = (double)p->nx * (double)p->ny * (double)p->nz;
    const double* kp[3] = {p->kp_d[0], p->kp_d[1], p->kp_d[2]};
    e = launch_coefs(p->tab, p->f32, (int)p->tab_e[0], (int)p->tab_e[1], (int)p->tab_e[2], (int)p->nx, (int)p->ny,
                     (int)p->nz, p->r[0], p->r[1], p->r[2], p->g0, p->d.c, p->d.dt, p->d.eps0, 1.0 / N, p->st,
                     p->order > 0 ? kp : nullptr);
    if (e != cudaSuccess) return cuda_fail(p, e, "coefficient table launch");
  }
  p->coeffs_ready = true;
  if (p->d.flags & PSATD_FLAG_AUTOTUNE) {
    bool cached = false;
    {
      std::lock_guard<std::mutex> lock(g_tune_mutex);
      const TuneKey key = tune_key(p);
      for (auto& kv : g_tune_cache)
        if (kv.first == key) {
          apply_cfg(p, kv.second);
          cached = true;
        }
    }
    if (cached) return regen_push_twiddles(p);
    return autotune(p, 5, nullptr);
  }
  return PSATD_OK;
}

psatd_status psatd_plan_autotune(psatd_plan p, int32_t reps, char* report, size_t report_len) {
  if (!p) return fail(nullptr, PSATD_ERR_INVALID_ARG, "plan is NULL");
  if (!p->coeffs_ready) return fail(p, PSATD_ERR_INVALID_ARG, "psatd_coeffs_init was not called");
  if (reps < 1 || reps > 1000) return fail(p, PSATD_ERR_INVALID_ARG, "reps must be in [1, 1000] (got %d)", reps);
  std::string rep;
  psatd_status s = autotune(p, reps, &rep);
  if (report && report_len > 0) {
    std::strncpy(report, rep.c_str(), report_len - 1);
    report[report_len - 1] = 0;
  }
  return s;
}

psatd_status psatd_plan_set_launch(psatd_plan p, const int32_t cfg[6]) {
  if (!p || !cfg) return fail(p, PSATD_ERR_INVALID_ARG, "plan or cfg is NULL");
  if (!p->coeffs_ready) return fail(p, PSATD_ERR_INVALID_ARG, "psatd_coeffs_init was not called");
  TuneSpace ts = tune_space(p);
  TuneCfg c{{-1, -1, -1, -1}, -1, push_ept((int)(p->ndim == 3 ? p->nz : p->ny), p->tc)};
  for (int k = 0; k < 4; ++k) {
    if (cfg[k] < 0) continue;
    if (cfg[k] > 30 || std::find(ts.rows[k].begin(), ts.rows[k].end(), cfg[k]) == ts.rows[k].end())
      return fail(p, PSATD_ERR_INVALID_ARG, "cfg[%d] = %d is not a valid launch shape of that pass", k, cfg[k]);
    c.log_tb[k] = cfg[k];
  }
  if (cfg[5] >= 0) {
    if (cfg[5] != 8 && cfg[5] != 16 && cfg[5] != 12 && cfg[5] != 20)
      return fail(p, PSATD_ERR_INVALID_ARG, "cfg[5] must be 8, 16, 12, 20 or -1");
    c.push_ept = cfg[5];
  }
  bool ok = false;
  for (auto& pt : ts.push) ok |= pt.ept == c.push_ept && (cfg[4] < 0 || pt.tb == cfg[4]);
  if (!ok) return fail(p, PSATD_ERR_INVALID_ARG, "fused pass: %d elements per thread and %d lines per CTA not valid",
                       c.push_ept, cfg[4]);
  c.push_tb = cfg[4];
  c.push_groups = p->cfg_push_groups;  // kept; psatd_plan_set_push_groups checks it against the new shape
  apply_cfg(p, c);
  return regen_push_twiddles(p);
}

psatd_status psatd_plan_set_push_groups(psatd_plan p, int32_t groups) {
  if (!p) return fail(nullptr, PSATD_ERR_INVALID_ARG, "plan is NULL");
  if (groups < 0) {
    p->cfg_push_groups = -1;
    return PSATD_OK;
  }
  const int64_t nlines = p->ndim == 3 ? p->nxh * p->ny : p->nxh * p->npatch;
  const int Ll = (int)(p->ndim == 3 ? p->nz : p->ny);
  const int tb = p->cfg_push_tb > 0 ? p->cfg_push_tb : push_lines_per_cta(Ll, p->n_in, nlines, p->tc, p->f32, p->push_ept);
  int maxsm = 0;
  cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, p->device);
  const size_t csz = p->f32 ? 8 : 16;
  const size_t smem = (p->tc ? (size_t)kTcTail : 0) + push_smem(p->n_in, Ll, tb, groups, csz, p->tc);
  if (!push_groups_ok(Ll, p->push_ept, tb, groups, p->tc, p->f32) || (maxsm > 0 && smem > (size_t)maxsm))
    return fail(p, PSATD_ERR_INVALID_ARG,
                "fused pass: %d component groups not valid with %d-point lines, %d elements per thread, "
                "%d lines per CTA and this precision",
                groups, Ll, p->push_ept, tb);
  p->cfg_push_groups = groups;
  return PSATD_OK;
}

psatd_status psatd_plan_get_push_groups(psatd_plan p, int32_t* groups) {
  if (!p || !groups) return fail(p, PSATD_ERR_INVALID_ARG, "plan or groups is NULL");
  const int64_t nlines = p->ndim == 3 ? p->nxh * p->ny : p->nxh * p->npatch;
  const int Ll = (int)(p->ndim == 3 ? p->nz : p->ny);
  const int tb = p->cfg_push_tb > 0 ? p->cfg_push_tb : push_lines_per_cta(Ll, p->n_in, nlines, p->tc, p->f32, p->push_ept);
  int G = p->cfg_push_groups > 0 ? p->cfg_push_groups
                                 : push_groups_default(Ll, p->push_ept, tb, p->n_in, p->tc, p->f32, p->f32 ? 8 : 16,
                                                       p->maxsm, p->sm_bytes);
  if (!push_groups_ok(Ll, p->push_ept, tb, G, p->tc, p->f32)) G = 1;
  *groups = G;
  return PSATD_OK;
}

psatd_status psatd_plan_get_launch(psatd_plan p, int32_t cfg[6]) {
  if (!p || !cfg) return fail(p, PSATD_ERR_INVALID_ARG, "plan or cfg is NULL");
  const int Lx = (int)(p->nx / 2);
  const int64_t nlines = p->ndim == 3 ? p->nxh * p->ny : p->nxh * p->npatch;
  const int Ll = (int)(p->ndim == 3 ? p->nz : p->ny);
  const bool tc = p->tc;
  const int dflt[4] = {pick_log_tb(Lx, p->ny, p->f32, tc, true),
                       p->ndim == 3 ? pick_log_tb((int)p->ny, p->nz, p->f32, tc) : -1,
                       p->ndim == 3 ? pick_log_tb_inv((int)p->ny, p->nz, p->f32, tc) : -1,
                       pick_log_tb_inv(Lx, p->ny, p->f32, tc)};
  for (int k = 0; k < 4; ++k) cfg[k] = p->cfg_log_tb[k] >= 0 ? p->cfg_log_tb[k] : dflt[k];
  cfg[4] = p->cfg_push_tb > 0 ? p->cfg_push_tb : push_lines_per_cta(Ll, p->n_in, nlines, p->tc, p->f32, p->push_ept);
  cfg[5] = p->push_ept;
  return PSATD_OK;
}

psatd_status psatd_step(psatd_plan p, const psatd_fields* fields, const psatd_sources* sources, int32_t nsteps) {
  NvtxRange range("psatd_step");
  if (!p) return fail(nullptr, PSATD_ERR_INVALID_ARG, "plan is NULL");
  if (nsteps < 1) return fail(p, PSATD_ERR_INVALID_ARG, "nsteps must be >= 1 (got %d)", nsteps);
  if (!p->coeffs_ready) return fail(p, PSATD_ERR_INVALID_ARG, "psatd_coeffs_init was not called");
  const void* in[kMaxComp] = {};
  void* out[kMaxComp] = {};
  psatd_status s = gather_slots(p, fields, sources, in, out);
  if (s != PSATD_OK) return s;
  for (int i = 0; i < nsteps; ++i) {
    s = step_once(p, in, out);
    if (s != PSATD_OK) return s;
  }
  return PSATD_OK;
}

psatd_status psatd_plan_sync(psatd_plan p) {
  if (!p) return fail(nullptr, PSATD_ERR_INVALID_ARG, "plan is NULL");
  cudaError_t e = cudaStreamSynchronize(p->st);
  if (e != cudaSuccess) return cuda_fail(p, e, "stream synchronise");
  e = cudaGetLastError();
  if (e != cudaSuccess) return cuda_fail(p, e, "asynchronous error");
  if (p->d_err) {
    int w = 0;
    e = cudaMemcpy(&w, p->d_err, sizeof w, cudaMemcpyDeviceToHost);
    if (e != cudaSuccess) return cuda_fail(p, e, "error word read");
    if (w != 0) {
      cudaMemset(p->d_err, 0, sizeof(int));
      if (w & kErrMmaWait)
        return fail(p, PSATD_ERR_TIMEOUT, "a tensor-core pass gave up waiting for its MMAs (error word %d)", w);
      if (w & kErrStageWait)
        return fail(p, PSATD_ERR_TIMEOUT, "the fused pass gave up waiting for its staged inputs (error word %d)", w);
      if (w & kErrBounds)
        return fail(p, PSATD_ERR_BOUNDS, "a pass's index check failed; its CTA skipped its accesses (error word %d)",
                    w);
      return fail(p, PSATD_ERR_NONFINITE, "NaN or Inf in a step's output since the last sync (error word %d)", w);
    }
  }
  return PSATD_OK;
}

psatd_status psatd_plan_destroy(psatd_plan p) {
  if (!p) return PSATD_OK;
  cudaStreamSynchronize(p->st);
  release(p);
  delete p;
  return PSATD_OK;
}

size_t psatd_plan_workspace_bytes(psatd_plan p) { return p ? p->bytes : 0; }

psatd_status psatd_plan_set_timing(psatd_plan p, int32_t enable) {
  if (!p) return fail(nullptr, PSATD_ERR_INVALID_ARG, "plan is NULL");
  cudaStreamSynchronize(p->st);
  for (auto& v : p->ev) {
    for (auto& e : v) p->pool.push_back(e);
    v.clear();
  }
  p->timing = enable != 0;
  return PSATD_OK;
}

int32_t psatd_kernel_times(psatd_plan p, int32_t n_slots, const char** names, int64_t* launches, double* total_ms) {
  if (!p) return 0;
  cudaStreamSynchronize(p->st);
  int used = 0;
  for (int s = 0; s < K_NSLOTS && used < n_slots; ++s) {
    if (p->ev[s].empty()) continue;
    double ms = 0;
    for (auto& e : p->ev[s]) {
      float t = 0;
      if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) ms += t;
      else cudaGetLastError();
    }
    if (names) names[used] = kSlotNames[s];
    if (launches) launches[used] = (int64_t)p->ev[s].size();
    if (total_ms) total_ms[used] = ms;
    ++used;
  }
  return used;
}

psatd_status fdtd_step(const psatd_desc* desc, int32_t scheme, const psatd_fields* fields,
                       const psatd_sources* sources, int32_t nsteps, void* cuda_stream) {
  NvtxRange range("fdtd_step");
  psatd_status s = validate_desc(nullptr, desc, false);
  if (s != PSATD_OK) return s;
  if (scheme != PSATD_FDTD_YEE && scheme != PSATD_FDTD_CKC)
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "unknown FDTD scheme %d", scheme);
  if (scheme == PSATD_FDTD_CKC && desc->ndim != 2)
    return fail(nullptr, PSATD_ERR_UNSUPPORTED, "the CKC scheme is provided in 2D only");
  if (desc->src == PSATD_SRC_J_RHO)
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "FDTD takes J only (src must be NONE or J)");
  if (nsteps < 1) return fail(nullptr, PSATD_ERR_INVALID_ARG, "nsteps must be >= 1 (got %d)", nsteps);
  if (!fields) return fail(nullptr, PSATD_ERR_INVALID_ARG, "fields is NULL");
  bool pe[3], pb[3], pj[3];
  present(desc->layout, pe, pb, pj);
  const void* J[3] = {nullptr, nullptr, nullptr};
  for (int i = 0; i < 3; ++i) {
    if (pe[i] != (fields->E[i] != nullptr) || pb[i] != (fields->B[i] != nullptr))
      return fail(nullptr, PSATD_ERR_INVALID_ARG, "field component %d presence does not match the layout", i);
    if ((fields->E[i] && !aligned16(fields->E[i])) || (fields->B[i] && !aligned16(fields->B[i])))
      return fail(nullptr, PSATD_ERR_INVALID_ARG, "field arrays must be 16-byte aligned");
  }
  int dev = 0;
  cudaGetDevice(&dev);
  for (int i = 0; i < 3; ++i)
    if ((fields->E[i] && !dev_accessible(fields->E[i], dev)) || (fields->B[i] && !dev_accessible(fields->B[i], dev)))
      return fail(nullptr, PSATD_ERR_INVALID_ARG, "field arrays must be accessible from the current device");
  if (desc->src == PSATD_SRC_J) {
    if (!sources) return fail(nullptr, PSATD_ERR_INVALID_ARG, "sources is NULL");
    for (int i = 0; i < 3; ++i) {
      if (pj[i] != (sources->J[i] != nullptr))
        return fail(nullptr, PSATD_ERR_INVALID_ARG, "J component %d presence does not match the layout", i);
      if (sources->J[i] && !aligned16(sources->J[i]))
        return fail(nullptr, PSATD_ERR_INVALID_ARG, "J arrays must be 16-byte aligned");
      if (sources->J[i] && !dev_accessible(sources->J[i], dev))
        return fail(nullptr, PSATD_ERR_INVALID_ARG, "J arrays must be accessible from the current device");
      J[i] = sources->J[i];
    }
  }
  const int64_t nz = desc->ndim == 3 ? desc->n[2] : 1;
  if (desc->n[1] > 65535 || nz > 65535) return fail(nullptr, PSATD_ERR_UNSUPPORTED, "ny, nz must be <= 65535");
  cudaStream_t st = static_cast<cudaStream_t>(cuda_stream);
  cudaError_t e = desc->prec == PSATD_FP32
                      ? launch_fdtd<float>(desc->ndim, scheme, desc->n[0], desc->n[1], nz, desc->d, desc->dt, desc->c,
                                           desc->eps0, fields->E, fields->B, J, nsteps, st)
                      : launch_fdtd<double>(desc->ndim, scheme, desc->n[0], desc->n[1], nz, desc->d, desc->dt, desc->c,
                                            desc->eps0, fields->E, fields->B, J, nsteps, st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "fdtd launch");
  return PSATD_OK;
}

psatd_status psatd_farfield(const psatd_desc* grid, const void* field, const int64_t window[4], int32_t apodise,
                            int32_t nk, const double* k, double* out, void* cuda_stream) {
  if (!grid || !field || !window || !k || !out)
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "grid, field, window, k and out must be non-NULL");
  if (grid->ndim != 2) return fail(nullptr, PSATD_ERR_UNSUPPORTED, "the far-field transform takes 2D fields");
  if (grid->prec != PSATD_FP32 && grid->prec != PSATD_FP64)
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "the field must be PSATD_FP32 or PSATD_FP64");
  const int64_t nx = grid->n[0], ny = grid->n[1];
  if (nx < 1 || ny < 1 || !pos_finite(grid->d[0]) || !pos_finite(grid->d[1]))
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "grid sizes must be >= 1 and cell sizes finite and > 0");
  const int64_t x0 = window[0], x1 = window[1], y0 = window[2], y1 = window[3];
  if (x0 < 0 || x1 > nx || x0 >= x1 || y0 < 0 || y1 > ny || y0 >= y1)
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "window [%lld, %lld) x [%lld, %lld) is empty or outside the grid",
                (long long)x0, (long long)x1, (long long)y0, (long long)y1);
  if (x1 - x0 > kFarfieldMaxRow)
    return fail(nullptr, PSATD_ERR_UNSUPPORTED, "window rows longer than %lld cells", (long long)kFarfieldMaxRow);
  if (apodise < 0 || apodise > 2) return fail(nullptr, PSATD_ERR_INVALID_ARG, "apodise must be 0, 1 or 2");
  if (nk < 1) return fail(nullptr, PSATD_ERR_INVALID_ARG, "nk must be >= 1");
  int dev = 0;
  cudaGetDevice(&dev);
  if (!dev_accessible(field, dev) || !dev_accessible(k, dev) || !dev_accessible(out, dev))
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "field, k and out must be accessible from the current device");
  const size_t esz = grid->prec == PSATD_FP32 ? 4 : 8;
  if ((reinterpret_cast<uintptr_t>(field) % esz) || (reinterpret_cast<uintptr_t>(k) % 8) ||
      (reinterpret_cast<uintptr_t>(out) % 8))
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "field, k or out misaligned for its element type");
  FarfieldArgs a;
  a.F = field;
  a.nx = nx;
  a.x0 = x0;
  a.x1 = x1;
  a.y0 = y0;
  a.y1 = y1;
  a.dx = grid->d[0];
  a.dy = grid->d[1];
  a.win_x = apodise >= 1;
  a.win_y = apodise == 2;
  a.k = k;
  a.out = out;
  a.nk = nk;
  cudaError_t e = launch_farfield(grid->prec == PSATD_FP32, a, static_cast<cudaStream_t>(cuda_stream));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "far-field launch");
  return PSATD_OK;
}

const char* psatd_last_error(psatd_plan p) { return p ? p->err.c_str() : g_err.c_str(); }

}  // extern "C"

// ---------------------------------------------------------------------------
// psatd_step_noalloc: the PSATD step for callers that cannot allocate device
// memory (see include/psatd.h).  Its scratch (spectra, twiddles, coefficient
// table) lives in one fixed, file-scope device array of kNoAllocBytes that
// every GPU loading this library holds until the process exits.
// ---------------------------------------------------------------------------
namespace {

constexpr size_t kNoAllocBytes = size_t(16) << 20;  // 16 MiB
static __device__ __align__(256) unsigned char g_noalloc_scratch[kNoAllocBytes];

constexpr int kNoAllocMaxDevices = 64;
// per device: the array's device address and the id of the context it was looked up in
void* g_noalloc_ptr[kNoAllocMaxDevices] = {};
unsigned long long g_noalloc_ctx[kNoAllocMaxDevices] = {};
std::mutex g_noalloc_mutex;

size_t round256(size_t v) { return (v + 255) & ~size_t(255); }

// Unique id of the calling thread's current CUDA context (driver entry points
// reached through the runtime, so the library needs no link against libcuda).
// A device reset destroys the context that the array was mapped in and the next
// runtime call creates a new one with a new id, so a cached address is looked up
// again.  Returns false when the id is not available (the caller then looks the
// address up on every call).
bool current_ctx_id(unsigned long long* id) {
  typedef int (*GetCurrentFn)(void**);
  typedef int (*GetIdFn)(void*, unsigned long long*);
  static GetCurrentFn get_current = nullptr;
  static GetIdFn get_id = nullptr;
  static bool resolved = false;
  if (!resolved) {  // called with g_noalloc_mutex held
    resolved = true;
    cudaDriverEntryPointQueryResult q1 = cudaDriverEntryPointSymbolNotFound, q2 = q1;
    void* f1 = nullptr;
    void* f2 = nullptr;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", &f1, 12000, cudaEnableDefault, &q1) == cudaSuccess &&
        cudaGetDriverEntryPointByVersion("cuCtxGetId", &f2, 12000, cudaEnableDefault, &q2) == cudaSuccess &&
        q1 == cudaDriverEntryPointSuccess && q2 == cudaDriverEntryPointSuccess) {
      get_current = reinterpret_cast<GetCurrentFn>(f1);
      get_id = reinterpret_cast<GetIdFn>(f2);
    }
    cudaGetLastError();
  }
  if (!get_current || !get_id) return false;
  void* ctx = nullptr;
  if (get_current(&ctx) != 0 || !ctx) return false;
  return get_id(ctx, id) == 0;
}

}  // namespace

extern "C" psatd_status psatd_step_noalloc(const psatd_desc* desc, const psatd_fields* fields,
                                           const psatd_sources* sources, int32_t nsteps, void* cuda_stream) {
  NvtxRange range("psatd_step_noalloc");
  psatd_status s = validate_desc(nullptr, desc, true);
  if (s != PSATD_OK) return s;
  if (nsteps < 1) return fail(nullptr, PSATD_ERR_INVALID_ARG, "nsteps must be >= 1 (got %d)", nsteps);
  if (desc->prec != PSATD_FP32 && desc->prec != PSATD_FP64)
    return fail(nullptr, PSATD_ERR_UNSUPPORTED, "psatd_step_noalloc runs PSATD_FP32 and PSATD_FP64 only");
  if (desc->order != 0)
    return fail(nullptr, PSATD_ERR_UNSUPPORTED, "psatd_step_noalloc runs the collocated exact-k step (order 0) only");
  if (desc->flags & PSATD_FLAG_CHECKED)
    return fail(nullptr, PSATD_ERR_UNSUPPORTED, "psatd_step_noalloc has no error word for PSATD_FLAG_CHECKED");

  // a plan-shaped descriptor on the stack whose buffers are carved from the array
  psatd_plan_s p;
  p.d = *desc;
  p.st = static_cast<cudaStream_t>(cuda_stream);
  cudaGetDevice(&p.device);
  p.f32 = desc->prec == PSATD_FP32;
  p.ndim = desc->ndim;
  p.layout = desc->layout;
  p.form = desc->src;
  counts(p.layout, p.form, &p.n_in, &p.n_out);
  p.nx = desc->n[0];
  p.ny = desc->n[1];
  p.nz = p.ndim == 3 ? desc->n[2] : 1;
  p.nxh = p.nx / 2 + 1;
  p.cs = p.nxh * p.ny * p.nz;
  p.push_ept = push_ept((int)(p.ndim == 3 ? p.nz : p.ny));
  const size_t csz = p.f32 ? 8 : 16;
  const int64_t ns[3] = {p.nx, p.ny, p.nz};
  p.tab_e[0] = p.nx / 2 + 1;
  p.tab_e[1] = p.ny / 2 + 1;
  p.tab_e[2] = p.ndim == 3 ? p.nz / 2 + 1 : 1;
  const size_t spec = round256((size_t)p.n_in * (size_t)p.cs * csz);
  size_t tw[3] = {0, 0, 0};
  for (int i = 0; i < p.ndim; ++i) tw[i] = round256((size_t)ns[i] * 16);
  const size_t tab = round256((size_t)p.tab_e[0] * p.tab_e[1] * p.tab_e[2] *
                              (p.f32 ? sizeof(Coef<float>) : sizeof(Coef<double>)));
  const size_t need = spec * (p.ndim == 3 ? 2 : 1) + tw[0] + tw[1] + tw[2] + tab;
  if (need > kNoAllocBytes)
    return fail(nullptr, PSATD_ERR_UNSUPPORTED,
                "psatd_step_noalloc: this grid needs %zu bytes of scratch, more than its fixed %zu-byte "
                "device array; use psatd_plan_create / psatd_step",
                need, kNoAllocBytes);

  int dev = 0;
  cudaError_t e = cudaGetDevice(&dev);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetDevice");
  if (dev < 0 || dev >= kNoAllocMaxDevices) return fail(nullptr, PSATD_ERR_UNSUPPORTED, "device index %d too large", dev);
  {
    int maxsm = 0;
    cudaDeviceGetAttribute(&maxsm, cudaDevAttrMaxSharedMemoryPerBlockOptin, dev);
    const int L = (int)(p.ndim == 3 ? p.nz : p.ny);
    const size_t smem = push_smem(p.n_in, L, 1, 1, csz);
    p.maxsm = maxsm;
    cudaDeviceGetAttribute(&p.sm_bytes, cudaDevAttrMaxSharedMemoryPerMultiprocessor, dev);
    if (maxsm > 0 && smem > (size_t)maxsm)
      return fail(nullptr, PSATD_ERR_UNSUPPORTED, "last-axis length %d needs %zu bytes of shared memory", L, smem);
  }
  const void* in[kMaxComp] = {};
  void* out[kMaxComp] = {};
  s = gather_slots(&p, fields, sources, in, out);  // also brings up the device's context
  if (s != PSATD_OK) {
    g_err = p.err;
    return s;
  }
  unsigned char* base = nullptr;
  {
    // set-up once per device and context (with that device current): the device address
    // of the array; a host-side reference to g_noalloc_scratch is not that address
    std::lock_guard<std::mutex> lock(g_noalloc_mutex);
    unsigned long long ctx = 0;
    const bool have_ctx = current_ctx_id(&ctx);
    if (!g_noalloc_ptr[dev] || !have_ctx || g_noalloc_ctx[dev] != ctx) {
      void* ptr = nullptr;
      e = cudaGetSymbolAddress(&ptr, g_noalloc_scratch);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "cudaGetSymbolAddress of the no-alloc scratch");
      g_noalloc_ptr[dev] = ptr;
      g_noalloc_ctx[dev] = have_ctx ? ctx : 0;
    }
    base = static_cast<unsigned char*>(g_noalloc_ptr[dev]);
  }
  size_t off = 0;
  p.spec1 = base + off;
  off += spec;
  if (p.ndim == 3) {
    p.spec2 = base + off;
    off += spec;
  }
  for (int i = 0; i < p.ndim; ++i) {
    p.tw[i] = base + off;
    off += tw[i];
  }
  p.tab = base + off;

  // wavenumber scale as in psatd_plan_create
  p.g0 = 2.0 * M_PI / ((double)p.nx * desc->d[0]);
  for (int i = 0; i < 3; ++i) {
    if (i >= p.ndim) {
      p.r[i] = 0.0;
      continue;
    }
    double ri = (2.0 * M_PI / ((double)ns[i] * desc->d[i])) / p.g0;
    if (p.f32) ri = (double)(float)ri;
    p.r[i] = ri;
  }
  // the tables are rebuilt by every call (the array keeps the previous call's contents);
  // the spectra need no clearing: the first pass overwrites them entirely
  for (int i = 0; i < p.ndim; ++i) {
    const int L = i == 0 ? (int)(ns[0] / 2) : (int)ns[i];
    const bool push_axis = (i == p.ndim - 1) && i > 0;
    e = launch_twiddles(p.tw[i], L, push_axis ? p.push_ept : row_ept(L), i == 0, p.f32, p.st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "twiddle table launch");
  }
  const double N = (double)p.nx * (double)p.ny * (double)p.nz;
  e = launch_coefs(p.tab, p.f32, (int)p.tab_e[0], (int)p.tab_e[1], (int)p.tab_e[2], (int)p.nx, (int)p.ny, (int)p.nz,
                   p.r[0], p.r[1], p.r[2], p.g0, desc->c, desc->dt, desc->eps0, 1.0 / N, p.st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "coefficient table launch");
  p.coeffs_ready = true;
  for (int i = 0; i < nsteps; ++i) {
    s = step_once(&p, in, out);
    if (s != PSATD_OK) {
      g_err = p.err;
      return s;
    }
  }
  return PSATD_OK;
}

// ---------------------------------------------------------------------------
// Batches of 2D patches (the paper's local-FFT subdomains, Sec. II.A.3): each
// patch is its own periodic domain; patches of one size form a class advanced
// with one launch per pass (patch index on the grid); a multi-step call is
// replayed from a CUDA graph of one step.
// ---------------------------------------------------------------------------
struct psatd_batch_s {
  cudaStream_t st = nullptr;
  int npatch = 0;
  bool f32 = true;
  std::vector<psatd_plan> cls;  // one plan per patch size class
  // The classes are independent (each plan has its own scratch): every step
  // forks from st into branch streams, each running its share of the classes
  // (balanced by cells), and joins back, so that the kernels of small classes
  // run beside those of other classes instead of one after another.
  std::vector<cudaStream_t> br;
  cudaEvent_t fork = nullptr;
  std::vector<cudaEvent_t> join;
  std::vector<int> branch_of;   // branch stream of each class when forked
  bool fork_on = true;          // psatd_batch_set_branches: forked (true) or one stream
  int64_t total_cells = 0;
  cudaGraph_t graph = nullptr;
  cudaGraphExec_t gexec = nullptr;
  const void* gkey[2 * kMaxComp] = {};
  // Persistent mode (persist.cuh): per pass type and length family (0 powers of two,
  // 1 the 3 * 2^k lengths) one launch over every class's work items.
  bool persist_ok = false;   // every class has lengths the persistent passes take
  bool persist = false;      // in use (psatd_batch_set_persistent; off by default)
  void* d_xf = nullptr;      // XClassArgs per class: x forward, x inverse
  void* d_xi = nullptr;
  void* d_push = nullptr;    // PushArgs<float> per class
  void* d_tws = nullptr;     // fused-axis twiddle table per class
  BatchItem* d_items = nullptr;
  unsigned* d_ctr = nullptr;  // two counters per queue
  struct Queue {
    int pass;       // 0 x forward, 1 fused, 2 x inverse
    int fam;
    int64_t first;  // offset of its items in d_items
    int n;
    int grid;
  };
  std::vector<Queue> queues;
  const void* pkey[2 * kMaxComp] = {};  // field / source pointers the x-pass arguments hold
  bool pkey_set = false;
};

namespace {

void batch_release(psatd_batch b) {
  void* bufs[] = {b->d_xf, b->d_xi, b->d_push, b->d_tws, b->d_items, b->d_ctr};
  for (void* q : bufs)
    if (q) cudaFree(q);
  b->d_xf = b->d_xi = b->d_push = b->d_tws = nullptr;
  b->d_items = nullptr;
  b->d_ctr = nullptr;
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  for (cudaStream_t s : b->br) cudaStreamDestroy(s);
  for (cudaEvent_t e : b->join) cudaEventDestroy(e);
  if (b->fork) cudaEventDestroy(b->fork);
  b->br.clear();
  b->join.clear();
  b->fork = nullptr;
  for (psatd_plan p : b->cls) {
    release(p);
    delete p;
  }
  b->cls.clear();
}

// ---- persistent mode
// the lengths of the persistent passes' case lists (persist.cuh)
bool persist_x_len(int L, bool tc) {
  return (pow2(L) && L >= 32 && L <= 512) || (!tc && three_pow2(L) && L >= 48 && L <= 384);
}
bool persist_y_len(int L, bool tc) {
  return (pow2(L) && L >= 64 && L <= 1024) || (!tc && three_pow2(L) && L >= 48 && L <= 768);
}
int fam_of(int L) { return pow2(L) ? 0 : 1; }
// rows per item of a transposing pass and lines per item of the fused pass
int persist_x_tb(int L) { return kPersistXThreads / (L / row_ept(L)); }
int persist_y_tb(int L, bool tc) { return kPersistThreads / (L / (pow2(L) ? (tc ? 16 : 8) : 12)); }

// X-pass arguments of class plan p for the step's field / source pointers (as
// run_step's first and last passes in 2D).
XClassArgs make_x_args(psatd_plan p, bool fwd, const void* in[kMaxComp], void* out[kMaxComp]) {
  XClassArgs a;
  std::memset(&a, 0, sizeof a);
  const bool chk = (p->d.flags & PSATD_FLAG_CHECKED) != 0;
  const int64_t shrink = (p->d.flags & PSATD_FLAG_TEST_SHORT_EXTENT) ? 1 : 0;
  const size_t csz = p->tc ? 8 : (p->f32 ? 8 : 16);
  char* s1 = static_cast<char*>(p->spec1);
  const int n = fwd ? p->n_in : p->n_out;
  for (int c = 0; c < n; ++c) {
    a.io.in[c] = fwd ? in[c] : static_cast<const void*>(s1 + c * p->cs * csz);
    a.io.out[c] = fwd ? static_cast<void*>(s1 + c * p->cs * csz) : out[c];
  }
  a.io.gmat = p->gmat;
  a.io.err = p->d_err;
  a.io.tc_ctl = (p->d.flags & PSATD_FLAG_TEST_STALL_MMA) ? kTcStallMma : 0;
  a.io.in_ext = chk ? (fwd ? p->caller_elems : p->cs) - shrink : 0;
  a.io.out_ext = chk ? (fwd ? p->cs : p->caller_elems) - shrink : 0;
  a.io.chk_err = p->d_err;
  a.tw = p->tw[0];
  if (fwd) {
    a.s0 = 0;                 // in_sa0 (patch offsets from the table)
    a.s1 = p->nx;             // in_sb
    a.s2 = p->nxh * p->ny;    // out_sa0
    a.s3 = p->ny;             // out_sk
  } else {
    a.s0 = p->nxh * p->ny;    // in_sa0
    a.s1 = p->ny;             // in_sk
    a.s2 = 0;                 // out_sa0
    a.s3 = p->nx;             // out_sb
  }
  a.off = p->d_off;
  a.nb = p->ny;
  a.L = (int)(p->nx / 2);
  return a;
}

// Build the persistent mode's tables (class arguments that do not depend on the
// step's pointers, work items, queues); leaves b->persist_ok false when a class
// has lengths the persistent passes do not take.
psatd_status persist_setup(psatd_batch b) {
  b->persist_ok = b->f32;
  for (psatd_plan p : b->cls)
    b->persist_ok = b->persist_ok && persist_x_len((int)(p->nx / 2), p->tc) && persist_y_len((int)p->ny, p->tc);
  if (!b->persist_ok) return PSATD_OK;
  const int ncls = (int)b->cls.size();
  const bool tc = b->cls[0]->tc;
  std::vector<PushArgs<float>> pa(ncls);
  std::vector<const void*> tws(ncls);
  for (int i = 0; i < ncls; ++i) {
    psatd_plan p = b->cls[i];
    pa[i] = make_push_args<float>(p, p->spec1, (int)p->ny, p->nxh * p->npatch);
    tws[i] = p->tw[1];
  }
  // work items, one queue per (pass, family), classes largest first
  std::vector<int> order(ncls);
  for (int i = 0; i < ncls; ++i) order[i] = i;
  std::stable_sort(order.begin(), order.end(), [&](int x, int y) {
    return b->cls[x]->nx * b->cls[x]->ny * b->cls[x]->npatch > b->cls[y]->nx * b->cls[y]->ny * b->cls[y]->npatch;
  });
  std::vector<BatchItem> items;
  b->queues.clear();
  for (int pass = 0; pass < 3; ++pass)
    for (int fam = 0; fam < 2; ++fam) {
      psatd_batch_s::Queue q{pass, fam, (int64_t)items.size(), 0, 0};
      for (int ci : order) {
        psatd_plan p = b->cls[ci];
        if (pass == 1) {
          const int L = (int)p->ny;
          if (fam_of(L) != fam) continue;
          const int tb = persist_y_tb(L, tc);
          const int64_t nl = p->nxh * p->npatch;
          for (int64_t blk = 0; blk < (nl + tb - 1) / tb; ++blk) items.push_back({ci, 0, 0, (int)blk});
        } else {
          const int L = (int)(p->nx / 2);
          if (fam_of(L) != fam) continue;
          const int tb = persist_x_tb(L);
          const int nc = pass == 0 ? p->n_in : p->n_out;
          const int64_t nblk = (p->ny + tb - 1) / tb;
          for (int a0 = 0; a0 < p->npatch; ++a0)
            for (int a1 = 0; a1 < nc; ++a1)
              for (int64_t blk = 0; blk < nblk; ++blk) items.push_back({ci, a0, a1, (int)blk});
        }
      }
      q.n = (int)(items.size() - q.first);
      if (q.n) b->queues.push_back(q);
    }
  cudaError_t e;
  auto dalloc = [&](void** ptr, size_t bytes) -> bool {
    e = cudaMalloc(ptr, bytes);
    if (e != cudaSuccess) {
      *ptr = nullptr;
      cudaGetLastError();
      return false;
    }
    return true;
  };
  if (!dalloc(&b->d_xf, ncls * sizeof(XClassArgs)) || !dalloc(&b->d_xi, ncls * sizeof(XClassArgs)) ||
      !dalloc(&b->d_push, ncls * sizeof(PushArgs<float>)) || !dalloc(&b->d_tws, ncls * sizeof(void*)) ||
      !dalloc(reinterpret_cast<void**>(&b->d_items), items.size() * sizeof(BatchItem)) ||
      !dalloc(reinterpret_cast<void**>(&b->d_ctr), 2 * b->queues.size() * sizeof(unsigned)))
    return fail(nullptr, PSATD_ERR_OOM, "batch persistent tables: %s", cudaGetErrorString(e));
  e = cudaMemcpy(b->d_push, pa.data(), ncls * sizeof(PushArgs<float>), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemcpy(b->d_tws, tws.data(), ncls * sizeof(void*), cudaMemcpyHostToDevice);
  if (e == cudaSuccess)
    e = cudaMemcpy(b->d_items, items.data(), items.size() * sizeof(BatchItem), cudaMemcpyHostToDevice);
  if (e == cudaSuccess) e = cudaMemset(b->d_ctr, 0, 2 * b->queues.size() * sizeof(unsigned));
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch persistent tables");
  // grids: the CTAs that stay resident together, at most the queue's chunks
  int nsm = 0, dev = 0;
  cudaGetDevice(&dev);
  cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, dev);
  const int layout = b->cls[0]->layout, n_in = b->cls[0]->n_in;
  const int tcv = tc ? (b->cls[0]->tc_bf16 ? 2 : 1) : 0;
  for (auto& q : b->queues) {
    int occ = 0;
    PersistQueue pq{nullptr, 0, nullptr};
    if (q.pass == 1) {
      if (tcv == 2) e = launch_persist_push<float, 2, 0>(layout, n_in, 0, b->st, nullptr, nullptr, pq, &occ);
      else if (tcv == 1) e = launch_persist_push<float, 1, 0>(layout, n_in, 0, b->st, nullptr, nullptr, pq, &occ);
      else if (q.fam == 0) e = launch_persist_push<float, 0, 0>(layout, n_in, 0, b->st, nullptr, nullptr, pq, &occ);
      else e = launch_persist_push<float, 0, 1>(layout, n_in, 0, b->st, nullptr, nullptr, pq, &occ);
    } else {
      const bool fwd = q.pass == 0;
      if (tcv == 2) e = launch_persist_x<float, 2, 0>(fwd, 0, b->st, nullptr, pq, &occ);
      else if (tcv == 1) e = launch_persist_x<float, 1, 0>(fwd, 0, b->st, nullptr, pq, &occ);
      else if (q.fam == 0) e = launch_persist_x<float, 0, 0>(fwd, 0, b->st, nullptr, pq, &occ);
      else e = launch_persist_x<float, 0, 1>(fwd, 0, b->st, nullptr, pq, &occ);
    }
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "persistent pass occupancy");
    const int chunks = (q.n + kPersistChunk - 1) / kPersistChunk;
    q.grid = std::max(1, std::min(chunks, std::max(occ, 1) * nsm));
  }
  // not the default: measured slower on the 512-patch workload (split-BF16 9.39 against 5.73 ms per
  // step, FP32 2.74 against 2.69), as a pass over the whole batch streams every class's spectra
  // through HBM where per-class launches run a class's three passes while its spectra are in L2
  b->persist = false;
  return PSATD_OK;
}

// Upload the x passes' class arguments when the step's pointers differ from the
// last upload (stream-ordered on the batch's stream, outside any capture).
psatd_status persist_upload(psatd_batch b, const void* in[kMaxComp], void* out[kMaxComp]) {
  const void* key[2 * kMaxComp];
  for (int i = 0; i < kMaxComp; ++i) {
    key[i] = in[i];
    key[kMaxComp + i] = out[i];
  }
  if (b->pkey_set && std::memcmp(key, b->pkey, sizeof key) == 0) return PSATD_OK;
  const int ncls = (int)b->cls.size();
  std::vector<XClassArgs> xf(ncls), xi(ncls);
  for (int i = 0; i < ncls; ++i) {
    xf[i] = make_x_args(b->cls[i], true, in, out);
    xi[i] = make_x_args(b->cls[i], false, in, out);
  }
  cudaError_t e = cudaMemcpyAsync(b->d_xf, xf.data(), ncls * sizeof(XClassArgs), cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess)
    e = cudaMemcpyAsync(b->d_xi, xi.data(), ncls * sizeof(XClassArgs), cudaMemcpyHostToDevice, b->st);
  if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);  // the host tables are freed on return
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch argument upload");
  std::memcpy(b->pkey, key, sizeof key);
  b->pkey_set = true;
  return PSATD_OK;
}

// One step of every class as one persistent launch per pass type and family.
psatd_status batch_launch_persist(psatd_batch b, void* out[kMaxComp]) {
  psatd_plan p0 = b->cls[0];
  const bool tc = p0->tc;
  const int tcv = tc ? (p0->tc_bf16 ? 2 : 1) : 0;
  const int slot[3] = {K_FWD_X, K_PUSH, K_INV_X};
  for (size_t qi = 0; qi < b->queues.size(); ++qi) {
    const auto& q = b->queues[qi];
    PersistQueue pq{b->d_items + q.first, q.n, b->d_ctr + 2 * qi};
    cudaError_t e;
    TimedLaunch tl(p0, slot[q.pass], b->st);
    if (q.pass == 1) {
      const PushArgs<float>* a = static_cast<const PushArgs<float>*>(b->d_push);
      const void* const* tws = static_cast<const void* const*>(b->d_tws);
      if (tcv == 2) e = launch_persist_push<float, 2, 0>(p0->layout, p0->n_in, q.grid, b->st, a, tws, pq);
      else if (tcv == 1) e = launch_persist_push<float, 1, 0>(p0->layout, p0->n_in, q.grid, b->st, a, tws, pq);
      else if (q.fam == 0) e = launch_persist_push<float, 0, 0>(p0->layout, p0->n_in, q.grid, b->st, a, tws, pq);
      else e = launch_persist_push<float, 0, 1>(p0->layout, p0->n_in, q.grid, b->st, a, tws, pq);
    } else {
      const bool fwd = q.pass == 0;
      const XClassArgs* a = static_cast<const XClassArgs*>(fwd ? b->d_xf : b->d_xi);
      if (tcv == 2) e = launch_persist_x<float, 2, 0>(fwd, q.grid, b->st, a, pq);
      else if (tcv == 1) e = launch_persist_x<float, 1, 0>(fwd, q.grid, b->st, a, pq);
      else if (q.fam == 0) e = launch_persist_x<float, 0, 0>(fwd, q.grid, b->st, a, pq);
      else e = launch_persist_x<float, 0, 1>(fwd, q.grid, b->st, a, pq);
    }
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "persistent batch pass launch");
  }
  if (p0->d.flags & PSATD_FLAG_CHECKED)
    for (psatd_plan p : b->cls) {
      cudaError_t e = launch_nonfinite(p->f32, out, p->n_out, p->d_off, p->npatch, p->nx * p->ny * p->nz, p->d_err,
                                       b->st);
      if (e != cudaSuccess) return cuda_fail(nullptr, e, "non-finite scan launch");
    }
  return PSATD_OK;
}

psatd_status batch_launch_all(psatd_batch b, const void* in[kMaxComp], void* out[kMaxComp]) {
  if (b->persist) return batch_launch_persist(b, out);
  const bool forked = !b->br.empty() && b->fork_on;
  cudaError_t e = cudaSuccess;
  if (forked) {
    e = cudaEventRecord(b->fork, b->st);
    for (size_t k = 0; k < b->br.size() && e == cudaSuccess; ++k) e = cudaStreamWaitEvent(b->br[k], b->fork, 0);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch fork");
  }
  for (psatd_plan p : b->cls) {
    psatd_status s = step_once(p, in, out);
    if (s != PSATD_OK) {
      g_err = p->err;
      return s;
    }
  }
  if (forked) {
    for (size_t k = 0; k < b->br.size() && e == cudaSuccess; ++k) {
      e = cudaEventRecord(b->join[k], b->br[k]);
      if (e == cudaSuccess) e = cudaStreamWaitEvent(b->st, b->join[k], 0);
    }
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "batch join");
  }
  return PSATD_OK;
}

}  // namespace

extern "C" psatd_status psatd_batch_create(const psatd_desc* base, int32_t npatch, const int64_t* n,
                                           void* cuda_stream, psatd_batch* out) {
  if (!out) return fail(nullptr, PSATD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!base) return fail(nullptr, PSATD_ERR_INVALID_ARG, "base desc is NULL");
  if (base->ndim != 2 || base->layout == PSATD_FIELDS_3D6)
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "batches hold 2D patches (layouts 2D6, TE, TM)");
  if (npatch < 1 || !n) return fail(nullptr, PSATD_ERR_INVALID_ARG, "npatch must be >= 1 and n non-NULL");
  std::vector<int64_t> off(npatch);
  std::vector<std::pair<int64_t, int64_t>> dims(npatch);
  int64_t acc = 0;
  for (int i = 0; i < npatch; ++i) {
    psatd_desc d = *base;
    d.n[0] = n[2 * i];
    d.n[1] = n[2 * i + 1];
    d.n[2] = 1;
    psatd_status s = validate_desc(nullptr, &d, true);
    if (s != PSATD_OK) {
      g_err = "patch " + std::to_string(i) + ": " + g_err;
      return s;
    }
    dims[i] = {d.n[0], d.n[1]};
    off[i] = acc;
    acc += d.n[0] * d.n[1];
  }
  psatd_batch b = new (std::nothrow) psatd_batch_s();
  if (!b) return fail(nullptr, PSATD_ERR_OOM, "host allocation failed");
  b->st = static_cast<cudaStream_t>(cuda_stream);
  b->npatch = npatch;
  b->f32 = base->prec != PSATD_FP64;
  b->total_cells = acc;
  std::vector<std::pair<int64_t, int64_t>> classes;
  for (auto& dd : dims)
    if (std::find(classes.begin(), classes.end(), dd) == classes.end()) classes.push_back(dd);
  for (auto& cl : classes) {
    std::vector<int64_t> offs;
    for (int i = 0; i < npatch; ++i)
      if (dims[i] == cl) offs.push_back(off[i]);
    psatd_desc d = *base;
    d.n[0] = cl.first;
    d.n[1] = cl.second;
    d.n[2] = 1;
    psatd_plan p = nullptr;
    psatd_status s = plan_create_n(&d, cuda_stream, (int)offs.size(), &p);
    if (s == PSATD_OK) {
      p->caller_elems = acc;  // the packed arrays of the whole batch
      s = alloc(p, reinterpret_cast<void**>(&p->d_off), offs.size() * sizeof(int64_t), "patch offsets");
      if (s == PSATD_OK) {
        cudaError_t e = cudaMemcpy(p->d_off, offs.data(), offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
        if (e != cudaSuccess) s = cuda_fail(p, e, "patch offset upload");
      }
      if (s == PSATD_OK) s = psatd_coeffs_init(p);
      if (s != PSATD_OK) g_err = p->err;
    }
    if (s != PSATD_OK) {
      if (p) {
        release(p);
        delete p;
      }
      batch_release(b);
      delete b;
      return s;
    }
    b->cls.push_back(p);
  }
  {  // persistent passes over every class, when all the classes' lengths allow them
    psatd_status s = persist_setup(b);
    if (s != PSATD_OK) {
      batch_release(b);
      delete b;
      return s;
    }
  }
  // branch streams: up to 4, classes assigned largest first to the least loaded branch
  const int nbr = (int)std::min<size_t>(4, b->cls.size());
  if (nbr > 1) {
    cudaError_t e = cudaEventCreateWithFlags(&b->fork, cudaEventDisableTiming);
    for (int k = 0; k < nbr && e == cudaSuccess; ++k) {
      cudaStream_t st = nullptr;
      cudaEvent_t ev = nullptr;
      e = cudaStreamCreateWithFlags(&st, cudaStreamNonBlocking);
      if (e == cudaSuccess) b->br.push_back(st);
      if (e == cudaSuccess) e = cudaEventCreateWithFlags(&ev, cudaEventDisableTiming);
      if (e == cudaSuccess) b->join.push_back(ev);
    }
    if (e == cudaSuccess) e = cudaStreamSynchronize(b->st);  // the classes' tables are built on st
    if (e != cudaSuccess) {
      psatd_status r = cuda_fail(nullptr, e, "batch branch streams");
      batch_release(b);
      delete b;
      return r;
    }
    std::vector<int> order(b->cls.size());
    for (size_t i = 0; i < order.size(); ++i) order[i] = (int)i;
    b->branch_of.assign(b->cls.size(), 0);
    auto cells = [&](int i) { return b->cls[i]->nx * b->cls[i]->ny * b->cls[i]->npatch; };
    std::stable_sort(order.begin(), order.end(), [&](int a, int c) { return cells(a) > cells(c); });
    std::vector<int64_t> load(nbr, 0);
    for (int i : order) {
      const int k = (int)(std::min_element(load.begin(), load.end()) - load.begin());
      load[k] += cells(i);
      b->cls[i]->st = b->br[k];
      b->branch_of[i] = k;
    }
  }
  *out = b;
  return PSATD_OK;
}

extern "C" psatd_status psatd_batch_step(psatd_batch b, const psatd_fields* fields, const psatd_sources* sources,
                                         int32_t nsteps) {
  NvtxRange range("psatd_batch_step");
  if (!b) return fail(nullptr, PSATD_ERR_INVALID_ARG, "batch is NULL");
  if (nsteps < 1) return fail(nullptr, PSATD_ERR_INVALID_ARG, "nsteps must be >= 1 (got %d)", nsteps);
  const void* in[kMaxComp] = {};
  void* out[kMaxComp] = {};
  psatd_status s = gather_slots(b->cls[0], fields, sources, in, out);
  if (s != PSATD_OK) {
    g_err = b->cls[0]->err;
    return s;
  }
  if (b->persist && (s = persist_upload(b, in, out)) != PSATD_OK) return s;
  if (nsteps == 1 || b->st == nullptr) {  // the legacy stream cannot be captured
    for (int i = 0; i < nsteps; ++i)
      if ((s = batch_launch_all(b, in, out)) != PSATD_OK) return s;
    return PSATD_OK;
  }
  const void* key[2 * kMaxComp];
  for (int i = 0; i < kMaxComp; ++i) {
    key[i] = in[i];
    key[kMaxComp + i] = out[i];
  }
  if (!b->gexec || std::memcmp(key, b->gkey, sizeof key) != 0) {
    if (b->gexec) cudaGraphExecDestroy(b->gexec);
    if (b->graph) cudaGraphDestroy(b->graph);
    b->gexec = nullptr;
    b->graph = nullptr;
    cudaError_t e = cudaStreamBeginCapture(b->st, cudaStreamCaptureModeThreadLocal);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "begin graph capture");
    s = batch_launch_all(b, in, out);
    cudaGraph_t g = nullptr;
    e = cudaStreamEndCapture(b->st, &g);
    if (s != PSATD_OK) {
      if (g) cudaGraphDestroy(g);
      return s;
    }
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "end graph capture");
    e = cudaGraphInstantiate(&b->gexec, g, 0);
    if (e != cudaSuccess) {
      cudaGraphDestroy(g);
      return cuda_fail(nullptr, e, "graph instantiate");
    }
    b->graph = g;
    std::memcpy(b->gkey, key, sizeof key);
  }
  for (int i = 0; i < nsteps; ++i) {
    cudaError_t e = cudaGraphLaunch(b->gexec, b->st);
    if (e != cudaSuccess) return cuda_fail(nullptr, e, "graph launch");
  }
  return PSATD_OK;
}

extern "C" int64_t psatd_batch_cells(psatd_batch b) { return b ? b->total_cells : 0; }

extern "C" psatd_status psatd_batch_set_persistent(psatd_batch b, int32_t enable) {
  if (!b) return fail(nullptr, PSATD_ERR_INVALID_ARG, "batch is NULL");
  if (enable && !b->persist_ok)
    return fail(nullptr, PSATD_ERR_UNSUPPORTED,
                "persistent passes need FP32 or mixed precision and sides whose line lengths they take "
                "(x: n/2 in 32..512 or 48..384 (3 * 2^k); last axis 64..1024 or 96..768)");
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "stream synchronise");
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->persist = enable != 0;
  return PSATD_OK;
}

extern "C" psatd_status psatd_batch_set_push_groups(psatd_batch b, int32_t groups) {
  if (!b) return fail(nullptr, PSATD_ERR_INVALID_ARG, "batch is NULL");
  if (groups == 0 || groups > 4 || groups == 3)
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "component groups must be 1, 2, 4 or -1 (got %d)", groups);
  cudaError_t e = cudaStreamSynchronize(b->st);
  for (cudaStream_t st : b->br)
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "stream synchronise");
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  for (psatd_plan p : b->cls)
    if (groups < 0 || psatd_plan_set_push_groups(p, groups) != PSATD_OK) p->cfg_push_groups = groups < 0 ? -1 : 1;
  return PSATD_OK;
}

extern "C" psatd_status psatd_batch_set_branches(psatd_batch b, int32_t forked) {
  if (!b) return fail(nullptr, PSATD_ERR_INVALID_ARG, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->st);
  for (cudaStream_t st : b->br)
    if (e == cudaSuccess) e = cudaStreamSynchronize(st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "stream synchronise");
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  b->fork_on = forked != 0;
  for (size_t i = 0; i < b->cls.size(); ++i)
    b->cls[i]->st = (b->fork_on && !b->br.empty()) ? b->br[b->branch_of[i]] : b->st;
  return PSATD_OK;
}

extern "C" int32_t psatd_batch_launches_per_step(psatd_batch b) {
  if (!b) return 0;
  if (b->persist) return (int32_t)b->queues.size();
  return (int32_t)(b->cls.size() * (b->cls.empty() ? 0 : 3));
}

extern "C" psatd_status psatd_batch_sync(psatd_batch b) {
  if (!b) return fail(nullptr, PSATD_ERR_INVALID_ARG, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "stream synchronise");
  for (psatd_plan p : b->cls) {
    psatd_status s = psatd_plan_sync(p);
    if (s != PSATD_OK) {
      g_err = p->err;
      return s;
    }
  }
  return PSATD_OK;
}

extern "C" psatd_status psatd_batch_set_timing(psatd_batch b, int32_t enable) {
  if (!b) return fail(nullptr, PSATD_ERR_INVALID_ARG, "batch is NULL");
  cudaError_t e = cudaStreamSynchronize(b->st);
  if (e != cudaSuccess) return cuda_fail(nullptr, e, "stream synchronise");
  // the event pairs are part of a recorded step graph: record it again
  if (b->gexec) cudaGraphExecDestroy(b->gexec);
  if (b->graph) cudaGraphDestroy(b->graph);
  b->gexec = nullptr;
  b->graph = nullptr;
  for (psatd_plan p : b->cls) {
    psatd_status s = psatd_plan_set_timing(p, enable);
    if (s != PSATD_OK) return s;
  }
  return PSATD_OK;
}

extern "C" int32_t psatd_batch_kernel_times(psatd_batch b, int32_t n_slots, const char** names, int64_t* launches,
                                            double* total_ms) {
  if (!b) return 0;
  cudaStreamSynchronize(b->st);
  int64_t nl[K_NSLOTS] = {};
  double ms[K_NSLOTS] = {};
  for (psatd_plan p : b->cls)
    for (int s = 0; s < K_NSLOTS; ++s)
      for (auto& e : p->ev[s]) {
        float t = 0;
        if (cudaEventElapsedTime(&t, e.a, e.b) == cudaSuccess) ms[s] += t;
        else cudaGetLastError();
        ++nl[s];
      }
  int used = 0;
  for (int s = 0; s < K_NSLOTS && used < n_slots; ++s) {
    if (!nl[s]) continue;
    if (names) names[used] = kSlotNames[s];
    if (launches) launches[used] = nl[s];
    if (total_ms) total_ms[used] = ms[s];
    ++used;
  }
  return used;
}

extern "C" psatd_status psatd_batch_destroy(psatd_batch b) {
  if (!b) return PSATD_OK;
  cudaStreamSynchronize(b->st);
  batch_release(b);
  delete b;
  return PSATD_OK;
}

// ---------------------------------------------------------------------------
// Local-FFT decomposition of one periodic 2D grid (Sec. II.A.3): patches with
// guard cells, refreshed from the neighbours every step, each advanced by its
// own FFTs (a batch of one size class), interiors written back.
// ---------------------------------------------------------------------------
struct psatd_local_s {
  psatd_plan plan = nullptr;  // px * py extended patches of one size
  cudaStream_t st = nullptr;
  int px = 1, py = 1, g = 0;
  int64_t nx = 0, ny = 0;
  void* fbuf = nullptr;       // packed extended patches, one array per input slot
  size_t comp_bytes = 0;
};

extern "C" psatd_status psatd_local_create(const psatd_desc* global, int32_t px, int32_t py, int32_t guard,
                                           void* cuda_stream, psatd_local* out) {
  if (!out) return fail(nullptr, PSATD_ERR_INVALID_ARG, "out is NULL");
  *out = nullptr;
  if (!global) return fail(nullptr, PSATD_ERR_INVALID_ARG, "desc is NULL");
  if (global->ndim != 2 || global->layout == PSATD_FIELDS_3D6)
    return fail(nullptr, PSATD_ERR_UNSUPPORTED, "the local decomposition is 2D (TE, TM, 2D6)");
  if (global->n[0] < 1 || global->n[1] < 1) return fail(nullptr, PSATD_ERR_INVALID_ARG, "grid sizes must be >= 1");
  psatd_status s;
  if (px < 1 || py < 1 || guard < 0) return fail(nullptr, PSATD_ERR_INVALID_ARG, "px, py >= 1 and guard >= 0 needed");
  if (global->n[0] % px || global->n[1] % py)
    return fail(nullptr, PSATD_ERR_INVALID_ARG, "px = %d, py = %d must divide the grid %lld x %lld", px, py,
                (long long)global->n[0], (long long)global->n[1]);
  psatd_desc pd = *global;
  pd.n[0] = global->n[0] / px + 2 * (int64_t)guard;
  pd.n[1] = global->n[1] / py + 2 * (int64_t)guard;
  s = validate_desc(nullptr, &pd, true);
  if (s != PSATD_OK) {
    g_err = "extended patch " + std::to_string(pd.n[0]) + " x " + std::to_string(pd.n[1]) + ": " + g_err;
    return s;
  }
  psatd_local L = new (std::nothrow) psatd_local_s();
  if (!L) return fail(nullptr, PSATD_ERR_OOM, "host allocation failed");
  L->st = static_cast<cudaStream_t>(cuda_stream);
  L->px = px;
  L->py = py;
  L->g = guard;
  L->nx = global->n[0];
  L->ny = global->n[1];
  const int npatch = px * py;
  s = plan_create_n(&pd, cuda_stream, npatch, &L->plan);
  psatd_plan p = L->plan;
  if (s == PSATD_OK) {
    std::vector<int64_t> offs(npatch);
    for (int i = 0; i < npatch; ++i) offs[i] = (int64_t)i * pd.n[0] * pd.n[1];
    s = alloc(p, reinterpret_cast<void**>(&p->d_off), offs.size() * sizeof(int64_t), "patch offsets");
    if (s == PSATD_OK) {
      cudaError_t e = cudaMemcpy(p->d_off, offs.data(), offs.size() * sizeof(int64_t), cudaMemcpyHostToDevice);
      if (e != cudaSuccess) s = cuda_fail(p, e, "patch offset upload");
    }
    L->comp_bytes = (size_t)npatch * pd.n[0] * pd.n[1] * (p->f32 ? 4 : 8);
    if (s == PSATD_OK) s = alloc(p, &L->fbuf, (size_t)p->n_in * L->comp_bytes, "patch fields");
    if (s == PSATD_OK) s = psatd_coeffs_init(p);
    if (s != PSATD_OK) g_err = p->err;
  }
  if (s != PSATD_OK) {
    if (L->fbuf) cudaFree(L->fbuf);
    if (p) {
      release(p);
      delete p;
    }
    delete L;
    return s;
  }
  *out = L;
  return PSATD_OK;
}

extern "C" psatd_status psatd_local_step(psatd_local L, const psatd_fields* fields, const psatd_sources* sources,
                                         int32_t nsteps) {
  NvtxRange range("psatd_local_step");
  if (!L) return fail(nullptr, PSATD_ERR_INVALID_ARG, "local decomposition is NULL");
  psatd_plan p = L->plan;
  if (nsteps < 1) return fail(p, PSATD_ERR_INVALID_ARG, "nsteps must be >= 1 (got %d)", nsteps);
  const void* in[kMaxComp] = {};
  void* out[kMaxComp] = {};
  psatd_status s = gather_slots(p, fields, sources, in, out);
  if (s != PSATD_OK) return s;
  const void* pin[kMaxComp] = {};
  void* pout[kMaxComp] = {};
  for (int c = 0; c < p->n_in; ++c) {
    pin[c] = static_cast<char*>(L->fbuf) + c * L->comp_bytes;
    if (c < p->n_out) pout[c] = const_cast<void*>(pin[c]);
  }
  LocalComps fc{}, sc{};
  for (int c = 0; c < p->n_out; ++c) {
    fc.global[c] = in[c];
    fc.global_out[c] = out[c];
    fc.patch[c] = pout[c];
  }
  for (int c = p->n_out; c < p->n_in; ++c) {
    sc.global[c - p->n_out] = in[c];
    sc.patch[c - p->n_out] = const_cast<void*>(pin[c]);
  }
  cudaError_t e;
  if (p->n_in > p->n_out) {  // sources: held constant over the call, refreshed once
    e = launch_guard_gather(p->f32, sc, p->n_in - p->n_out, L->nx, L->ny, L->px, L->py, L->g, p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "guard gather (sources)");
  }
  for (int i = 0; i < nsteps; ++i) {
    e = launch_guard_gather(p->f32, fc, p->n_out, L->nx, L->ny, L->px, L->py, L->g, p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "guard gather");
    if ((s = step_once(p, pin, pout)) != PSATD_OK) return s;
    e = launch_guard_scatter(p->f32, fc, p->n_out, L->nx, L->ny, L->px, L->py, L->g, p->st);
    if (e != cudaSuccess) return cuda_fail(p, e, "guard scatter");
  }
  return PSATD_OK;
}

extern "C" psatd_plan psatd_local_plan(psatd_local L) { return L ? L->plan : nullptr; }

extern "C" psatd_status psatd_local_destroy(psatd_local L) {
  if (!L) return PSATD_OK;
  cudaStreamSynchronize(L->st);
  if (L->fbuf) cudaFree(L->fbuf);
  if (L->plan) {
    release(L->plan);
    delete L->plan;
  }
  delete L;
  return PSATD_OK;
}
