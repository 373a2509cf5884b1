// C ABI of the AccAltProj library (include/rpca.h): context, workspace and the host loop
// that enqueues the fused pass and the tall-skinny kernel.
#include <cuda.h>
#include <cudaTypedefs.h>
#include <math.h>
#include <stdlib.h>
#include <string.h>

#include <algorithm>
#include <mutex>
#include <new>
#include <vector>

#include "../../include/rpca.h"
#include "common.cuh"
#include "mlp.cuh"
#include "tc_images.cuh"

namespace rpca {
unsigned long long g_attr_epoch = 1;  // see common.cuh
}  // namespace rpca

namespace rpca {
cudaError_t launch_pass_f32(int R, const PassArgs& a, cudaStream_t s);
cudaError_t launch_pass_f64(int R, const PassArgs& a, cudaStream_t s);
cudaError_t launch_extract_count_f32(int R, const ExtractArgs& a, cudaStream_t s);
cudaError_t launch_extract_count_f64(int R, const ExtractArgs& a, cudaStream_t s);
cudaError_t launch_extract_write_f32(int R, const ExtractArgs& a, cudaStream_t s);
cudaError_t launch_extract_write_f64(int R, const ExtractArgs& a, cudaStream_t s);
PassGeom pass_geometry_f32(int R);
PassGeom pass_geometry_f64(int R);

PassGeom pass_geometry(int prec, int R) { return prec == PREC_F32 ? pass_geometry_f32(R) : pass_geometry_f64(R); }
cudaError_t launch_fused_pass(int prec, int R, const PassArgs& a, cudaStream_t s) {
  return prec == PREC_F32 ? launch_pass_f32(R, a, s) : launch_pass_f64(R, a, s);
}
cudaError_t launch_extract_count(int prec, int R, const ExtractArgs& a, cudaStream_t s) {
  return prec == PREC_F32 ? launch_extract_count_f32(R, a, s) : launch_extract_count_f64(R, a, s);
}
cudaError_t launch_extract_write(int prec, int R, const ExtractArgs& a, cudaStream_t s) {
  return prec == PREC_F32 ? launch_extract_write_f32(R, a, s) : launch_extract_write_f64(R, a, s);
}
}  // namespace rpca

using namespace rpca;

struct rpca_ctx {
  rpca_params p;
  cudaStream_t stream = nullptr;
  int device = 0, small_grid = 0;
  int prec = PREC_F32;
  size_t tsize = 4;
  int64_t m = 0, n = 0, ld = 0;
  int r = 0, Rr = 0, b = 0, Rb = 0;
  const void* D = nullptr;
  void* Down = nullptr;
  int vec = 0;
  // bf16 storage of D (BF16 modes): hi part, then lo part (split mode), rows of ldb elements
  int dmode = 0;
  bool split = false;
  void* Dhl = nullptr;
  int64_t ldb = 0;
  // workspace
  // tall-skinny arrays in the working precision (tsize bytes per entry)
  void *U = nullptr, *sig = nullptr, *V = nullptr, *Ut = nullptr, *Vt = nullptr, *Y1 = nullptr, *Y2 = nullptr,
       *part = nullptr;
  void *Wc = nullptr, *Vc = nullptr, *Utc = nullptr, *Vtc = nullptr, *P1 = nullptr, *P2 = nullptr;
  double* resP = nullptr;
  unsigned long long* nnzP = nullptr;
  DevState* st = nullptr;
  DevStats* stats = nullptr;
  int* h_flags = nullptr;  // pinned: k, done, status, conv, use_lo, emit, emit_k, steps_run
  unsigned long long *rowcnt = nullptr, *rowoff = nullptr;
  bool ready = false;
  // learned threshold schedule: network parameters (mlp.cuh), unrolled depth, support
  // bitmasks of the last two passes and per-CTA support-change counts
  float* theta = nullptr;
  int depth = 0;
  bool theta_set = false;
  unsigned* masks = nullptr;
  long long mask_wr = 0, mask_words = 0;  // words per row (SIMT layout), words per buffer
  unsigned long long* chgP = nullptr;
  unsigned long long* obs_count = nullptr;  // partial observation: observed entries of D
  // tensor-core pass
  bool tc_iter = false, tc_init = false;
  CUtensorMap dmap, dmap_lo;
  int TR = 0, TC = 0;
  TcPlan plan;                 // tile partition of the tensor-core pass
  int4* d_rect = nullptr;      // its tables on the device
  int4* d_ids = nullptr;
  int* d_p1nsl = nullptr;
  float* tfac = nullptr;  // T_u, T_v from the tensor-core pass for the update (TcPassArgs)
  unsigned* swords = nullptr;  // support words of the last pass predicted to be final (TcPassArgs)
  unsigned* wcc = nullptr;     // support counts per row and chunk of support words
  long long last_nnz = -1;     // support count of the pass at iterate last_nnz_k (host copy)
  int last_nnz_k = -1;
  int last_iters = 0;          // iterations the last solve to its end took
  // operand images: set 0 read by the initialisation's pass, set 1 by the iteration's
  uint8_t *wop[2] = {nullptr, nullptr}, *vop[2] = {nullptr, nullptr}, *vtop[2] = {nullptr, nullptr},
          *utop[2] = {nullptr, nullptr};
  // allocation signature of the current workspace
  int64_t ws_m = -1, ws_n = -1;
  int ws_r = -1;
  // profiling: every launch (stride 1) or every stride-th fused pass only (stride > 1)
  bool prof = false;
  int prof_stride = 1;
  std::vector<cudaEvent_t> ev_free;
  // profiling timeline: events at the boundaries of timed launches (a kernel's end event is
  // the next kernel's begin event while nothing else was queued in between) and the intervals
  // {begin index, end index, is-pass, pass ordinal in the window} between them
  struct Span {
    int b, e;
    bool pass;
    int64_t ord;
  };
  std::vector<cudaEvent_t> ev_line;
  std::vector<Span> spans;
  bool line_open = false, cur_timed = false;
  int64_t win_pass = 0, win_other = 0;  // launches queued since the last collection
  int64_t pass_seq = 0;                 // pass launches since profiling was switched on
  double pass_ms = 0, other_ms = 0;
  int64_t pass_n = 0, other_n = 0;
};

namespace {

#define CK(call)                                 \
  do {                                           \
    cudaError_t e_ = (call);                     \
    if (e_ != cudaSuccess) return RPCA_ERR_CUDA; \
  } while (0)

void free_workspace(rpca_ctx* c) {
  void** ptrs[] = {&c->U,   &c->sig,  &c->V,    &c->Ut,   &c->Vt,
                   &c->Y1,  &c->Y2,   &c->part, &c->Wc,           &c->Vc,
                   &c->Utc,         &c->Vtc,          &c->P1,           &c->P2,           (void**)&c->resP,
                   (void**)&c->nnzP, (void**)&c->st, (void**)&c->stats, (void**)&c->rowcnt, (void**)&c->rowoff,
                   &c->Down, &c->Dhl, (void**)&c->wop[0], (void**)&c->vop[0], (void**)&c->vtop[0],
                   (void**)&c->utop[0], (void**)&c->wop[1], (void**)&c->vop[1], (void**)&c->vtop[1],
                   (void**)&c->utop[1], (void**)&c->masks, (void**)&c->chgP,
                   (void**)&c->d_rect, (void**)&c->d_ids, (void**)&c->d_p1nsl, (void**)&c->tfac,
                   (void**)&c->swords, (void**)&c->wcc};
  for (void** p : ptrs) {
    if (*p) cudaFree(*p);
    *p = nullptr;
  }
  c->ready = false;
}

cudaEvent_t take_event(rpca_ctx* c) {
  if (!c->ev_free.empty()) {
    cudaEvent_t e = c->ev_free.back();
    c->ev_free.pop_back();
    return e;
  }
  cudaEvent_t e = nullptr;
  cudaEventCreate(&e);
  return e;
}

// Marks the start (begin = true) or the end of one launch.  Every launch is counted; the
// timed ones get events at their boundaries.
void prof_mark(rpca_ctx* c, bool pass, bool begin) {
  if (!c->prof) return;
  if (begin) {
    const int64_t ord = pass ? c->win_pass++ : -1;
    if (!pass) ++c->win_other;
    c->cur_timed = c->prof_stride <= 1 || (pass && c->pass_seq % c->prof_stride == 0);
    if (pass) ++c->pass_seq;
    if (!c->cur_timed) {
      c->line_open = false;
      return;
    }
    if (!c->line_open) {
      cudaEvent_t e = take_event(c);
      cudaEventRecord(e, c->stream);
      c->ev_line.push_back(e);
    }
    c->spans.push_back({(int)c->ev_line.size() - 1, -1, pass, ord});
  } else {
    if (!c->cur_timed) return;
    cudaEvent_t e = take_event(c);
    cudaEventRecord(e, c->stream);
    c->ev_line.push_back(e);
    c->spans.back().e = (int)c->ev_line.size() - 1;
    c->line_open = true;
  }
}

// Something other than a profiled launch was queued (or the host waited): the next launch
// starts a new span.
void prof_break(rpca_ctx* c) { c->line_open = false; }

// Accumulates the recorded spans (the stream must be synchronised).  Only the first
// `effective_pass` pass launches of the window count as passes: pass launches past that count
// returned at once on the device and are counted with the other kernels, so the pass average
// covers only passes that did work.  Launches that were not timed add to the other count.
void prof_collect(rpca_ctx* c, int64_t effective_pass) {
  int64_t counted = 0;
  for (const auto& sp : c->spans) {
    if (sp.e < 0) continue;
    float t = 0.f;
    cudaEventElapsedTime(&t, c->ev_line[sp.b], c->ev_line[sp.e]);
    if (sp.pass && (effective_pass < 0 || sp.ord < effective_pass)) {
      c->pass_ms += t;
      ++c->pass_n;
      ++counted;
    } else {
      c->other_ms += t;
    }
  }
  c->other_n += c->win_pass + c->win_other - counted;
  c->win_pass = c->win_other = 0;
  for (cudaEvent_t e : c->ev_line) c->ev_free.push_back(e);
  c->ev_line.clear();
  c->spans.clear();
  c->line_open = false;
}

struct Grid {
  int n_p1, n_p2, n_cta;
};
bool use_tc(const rpca_ctx* c, int R) { return (R == c->Rr) ? c->tc_iter : (R == c->Rb ? c->tc_init : false); }

bool learned(const rpca_ctx* c) { return c->p.zeta_mode == RPCA_ZETA_LEARNED; }

Grid pass_grid(const rpca_ctx* c, int R) {
  if (use_tc(c, R)) return Grid{c->plan.Bmax, c->plan.S2, c->plan.ncta};
  const PassGeom g = pass_geometry(c->prec, R);
  const int gx = (int)((c->n + g.BW - 1) / g.BW), gy = (int)((c->m + g.BH - 1) / g.BH);
  return Grid{gx, gy, gx * gy};
}

// One fused pass at compiled rank R: the initialisation's (init) or the iteration's.
int run_pass(rpca_ctx* c, int R, bool init) {
  PassArgs a{};
  a.D = c->D;
  a.ld = c->ld;
  a.m = (int)c->m;
  a.n = (int)c->n;
  a.W = c->Wc;
  a.V = c->Vc;
  a.Ut = c->Utc;
  a.Vt = c->Vtc;
  a.st = c->st;
  a.P1 = c->P1;
  a.P2 = c->P2;
  a.resP = c->resP;
  a.nnzP = c->nnzP;
  a.vec = c->vec;
  a.dm = 0;
  a.Dlo = nullptr;
  if (c->dmode) {
    a.D = c->Dhl;
    a.ld = c->ldb;
    a.dm = 1;
    a.Dlo = c->split ? static_cast<const uint8_t*>(c->Dhl) + (size_t)c->m * c->ldb * 2 : nullptr;
  }
  // the learned schedule's support-change statistic: bitmasks in the iteration's passes
  const bool track = learned(c) && !init;
  a.masks = track ? c->masks : nullptr;
  a.mask_wr = c->mask_wr;
  a.mask_words = c->mask_words;
  a.chgP = track ? c->chgP : nullptr;
  a.partial = c->p.observed == RPCA_OBS_NAN ? 1 : 0;
  prof_mark(c, true, true);
  if (init ? c->tc_init : c->tc_iter) {
    TcPassArgs t{};
    t.m = (int)c->m;
    t.n = (int)c->n;
    t.R = R;
    t.ncta = c->plan.ncta;
    t.rect = c->d_rect;
    t.ids = c->d_ids;
    t.TR = c->TR;
    t.TC = c->TC;
    const int set = init ? 0 : 1;
    t.wop = c->wop[set];
    t.vop = c->vop[set];
    t.vtop = c->vtop[set];
    t.utop = c->utop[set];
    t.st = c->st;
    t.status = &c->st->status;
    t.P1 = static_cast<float*>(c->P1);
    t.P2 = static_cast<float*>(c->P2);
    t.resP = c->resP;
    t.nnzP = c->nnzP;
    t.masks = a.masks;
    t.mask_wr = c->mask_words;
    t.chgP = a.chgP;
    t.partial = a.partial;
    t.swords = (!init && !c->dmode && !track) ? c->swords : nullptr;  // not with the learned masks
    t.nw = 2 * c->TC;
    t.emit_k = &c->st->emit_k;
    t.tgram = static_cast<const float*>(c->part);
    t.tnb = c->small_grid;
    t.tw = c->r;
    t.tcta = c->plan.min_cta;
    t.tfac = init ? nullptr : c->tfac;
    CK(launch_fused_pass_tc(&c->dmap, &c->dmap_lo, c->dmode, t, c->stream));
    if (t.masks)  // the support changes since the previous pass, one count per CTA of the pass
      CK(launch_count_mask_changes(c->masks, c->mask_words, 256ll * c->TR * c->TC, c->st, c->chgP, c->plan.ncta,
                                   c->stream));
  } else {
    CK(launch_fused_pass(c->prec, R, a, c->stream));
  }
  prof_mark(c, true, false);
  return RPCA_OK;
}

int run_small(rpca_ctx* c, const SmallArgs& a) {
  prof_mark(c, false, true);
  CK(launch_small(a, c->small_grid, c->stream));
  prof_mark(c, false, false);
  return RPCA_OK;
}


// Tile partition of the tensor-core pass.  The TR x TC tiles (128 x 64) are cut into row
// groups of different heights; group g of h_g row tiles splits all TC column tiles among its
// own B_g CTAs (ranges of nearly equal width, at most max_ct column tiles each: the
// tensor-memory budget).  The plan takes the smallest largest-CTA cost (h (w + 1/2) for h row
// tiles of w column tiles) for which the groups fit on nsm CTAs (one per SM), and among those
// the one with the fewest partial products (every CTA writes an m-slice of Y1 for its rows and
// every group two n-slices of Y2).  Dynamic programming over (row tiles, CTAs).
bool tc_plan(int TR, int TC, int nsm, int max_ct, TcPlan* out) {
  if (TR < 1 || TC < 1 || nsm < 1) return false;
  const long long tiles = (long long)TR * TC;
  // cost of a CTA of h row tiles and w column tiles: h (w + 1/2) tile times (each new row tile
  // loads its W and U~ images and drains Y1: measured, a plan of one column tile per CTA ran at
  // half the bandwidth); T2 = twice the cost bound
  for (long long T2 = 2 * ((tiles + nsm - 1) / nsm); T2 <= 2 * tiles + 2 * TR; ++T2) {
    std::vector<std::pair<int, int>> opts;  // (group height, CTAs)
    for (int h = 1; h <= TR; ++h) {
      const long long w = std::min<long long>(std::min<long long>((T2 - h) / (2 * h), max_ct), TC);
      if (w < 1) continue;
      opts.push_back({h, (int)((TC + w - 1) / w)});
    }
    const double INF = 1e300;
    std::vector<double> best((size_t)(TR + 1) * (nsm + 1), INF);
    std::vector<int> pick((size_t)(TR + 1) * (nsm + 1), -1);
    auto at = [&](int rows, int c) { return (size_t)rows * (nsm + 1) + c; };
    best[at(0, 0)] = 0.0;
    for (int rows = 1; rows <= TR; ++rows)
      for (int o = 0; o < (int)opts.size(); ++o) {
        const int h = opts[o].first, B = opts[o].second;
        if (h > rows) break;
        for (int c = B; c <= nsm; ++c) {
          const double prev = best[at(rows - h, c - B)];
          if (prev >= INF) continue;
          const double v = prev + (double)h * 128.0 * B + (double)TC * 64.0;
          if (v < best[at(rows, c)]) {
            best[at(rows, c)] = v;
            pick[at(rows, c)] = o;
          }
        }
      }
    int cbest = -1;
    for (int c = 1; c <= nsm; ++c)
      if (best[at(TR, c)] < INF && (cbest < 0 || best[at(TR, c)] < best[at(TR, cbest)])) cbest = c;
    if (cbest < 0) continue;
    // unwind: groups from the bottom row tile up
    std::vector<std::pair<int, int>> groups;
    for (int rows = TR, c = cbest; rows > 0;) {
      const auto g = opts[pick[at(rows, c)]];
      groups.push_back(g);
      rows -= g.first;
      c -= g.second;
    }
    std::reverse(groups.begin(), groups.end());
    out->rect.clear();
    out->ids.clear();
    out->p1_nsl.assign(TR, 0);
    out->A = (int)groups.size();
    out->Bmax = 0;
    out->ct_max = 0;
    out->S2 = 0;
    int rt = 0;
    for (int gi = 0; gi < (int)groups.size(); ++gi) {
      const int h = groups[gi].first, B = groups[gi].second;
      for (int b = 0; b < B; ++b) {
        const int c0 = (int)((long long)b * TC / B), c1 = (int)((long long)(b + 1) * TC / B);
        out->rect.push_back(make_int4(rt, rt + h, c0, c1));
        out->ids.push_back(make_int4(gi, b, 2 * gi, 0));
        out->ct_max = std::max(out->ct_max, c1 - c0);
      }
      for (int q = rt; q < rt + h; ++q) out->p1_nsl[q] = B;
      out->Bmax = std::max(out->Bmax, B);
      out->S2 += 2;
      rt += h;
    }
    out->ncta = (int)out->rect.size();
    out->min_cta = 0;
    for (int i = 1; i < out->ncta; ++i) {
      const int4 a = out->rect[i], b = out->rect[out->min_cta];
      if ((a.y - a.x) * (a.w - a.z) < (b.y - b.x) * (b.w - b.z)) out->min_cta = i;
    }
    out->T = (int)(T2 / 2);
    return out->ct_max <= max_ct;
  }
  return false;
}

// Tensor map of an m x n row-major matrix with rows of `ld` elements, in boxes of 128 rows x
// 128 bytes (32 FP32 or 64 bf16 elements) with the 128-byte swizzle.
bool encode_map(CUtensorMap* map, const void* base, int64_t m, int64_t n, int64_t ld, bool bf16) {
  static PFN_cuTensorMapEncodeTiled_v12000 enc = nullptr;
  if (!enc) {
    cudaDriverEntryPointQueryResult q;
    if (cudaGetDriverEntryPointByVersion("cuTensorMapEncodeTiled", (void**)&enc, 12000, cudaEnableDefault, &q) !=
            cudaSuccess ||
        !enc)
      return false;
  }
  const int es_bytes = bf16 ? 2 : 4;
  cuuint64_t gdim[2] = {(cuuint64_t)n, (cuuint64_t)m};
  cuuint64_t gstr[1] = {(cuuint64_t)(ld * es_bytes)};
  cuuint32_t box[2] = {(cuuint32_t)(128 / es_bytes), 128}, es[2] = {1, 1};
  return enc(map, bf16 ? CU_TENSOR_MAP_DATA_TYPE_BFLOAT16 : CU_TENSOR_MAP_DATA_TYPE_FLOAT32, 2,
             const_cast<void*>(base), gdim, gstr, box, es, CU_TENSOR_MAP_INTERLEAVE_NONE, CU_TENSOR_MAP_SWIZZLE_128B,
             CU_TENSOR_MAP_L2_PROMOTION_L2_256B, CU_TENSOR_MAP_FLOAT_OOB_FILL_NONE) == CUDA_SUCCESS;
}

// D as the tensor-core pass reads it: FP32 D, or the bf16 hi / lo parts.
bool encode_dmap(rpca_ctx* c) {
  if (!c->dmode) return encode_map(&c->dmap, c->D, c->m, c->n, c->ld, false);
  const size_t part = (size_t)c->m * c->ldb * 2;
  const void* lo = c->split ? static_cast<const void*>(static_cast<const uint8_t*>(c->Dhl) + part) : c->Dhl;
  return encode_map(&c->dmap, c->Dhl, c->m, c->n, c->ldb, true) &&
         encode_map(&c->dmap_lo, lo, c->m, c->n, c->ldb, true);
}

SmallArgs small_args(rpca_ctx* c, int mode, int R) {
  SmallArgs a;
  memset(&a, 0, sizeof(a));
  const Grid g = pass_grid(c, R);
  a.mode = mode;
  a.m = (int)c->m;
  a.n = (int)c->n;
  a.r = c->r;
  a.R = R;
  a.b = c->b;
  a.prec = c->prec;
  a.n_p1 = g.n_p1;
  a.n_p2 = g.n_p2;
  a.p1_nsl = use_tc(c, R) ? c->d_p1nsl : nullptr;
  a.R2 = use_tc(c, R) ? tc_image_rank(R) : R;
  a.emit_ok = (c->swords && c->tc_iter && !c->dmode && !learned(c)) ? 1 : 0;
  a.tfac = (mode == SM_UPDATE && c->tc_iter) ? c->tfac : nullptr;
  a.n_cta = g.n_cta;
  a.P1 = c->P1;
  a.P2 = c->P2;
  a.resP = c->resP;
  a.nnzP = c->nnzP;
  a.chgP = (learned(c) && mode == SM_UPDATE) ? c->chgP : nullptr;
  a.theta = c->theta;
  a.depth = c->depth;
  a.U = c->U;
  a.sig = c->sig;
  a.V = c->V;
  a.Ut = c->Ut;
  a.Vt = c->Vt;
  a.Y1 = c->Y1;
  a.Y2 = c->Y2;
  a.part = c->part;
  a.Wc = c->Wc;
  a.Vc = c->Vc;
  a.Utc = c->Utc;
  a.Vtc = c->Vtc;
  a.Rc = c->Rb;
  a.Rit = c->Rr;
  a.st = c->st;
  a.stats = c->stats;
  a.init_tol = c->p.init_tol;
  a.init_max = c->p.init_max_passes;
  a.seed = 0x243f6a8885a308d3ull;
  for (int set = 0; set < 2; ++set) {
    a.wop[set] = c->wop[set];
    a.vop[set] = c->vop[set];
    a.vtop[set] = c->vtop[set];
    a.utop[set] = c->utop[set];
  }
  a.img_rk[0] = tc_image_rank(c->Rb);
  a.img_rk[1] = tc_image_rank(c->Rr);
  a.img_init = c->tc_init ? 1 : 0;
  a.img_iter = c->tc_iter ? 1 : 0;
  return a;
}

int read_flags(rpca_ctx* c) {
  prof_break(c);
  CK(cudaMemcpyAsync(c->h_flags, &c->st->k, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  return RPCA_OK;
}
// DevState layout: k, done, status, conv, use_lo, emit, emit_k, steps_run are consecutive ints.
inline int flag_k(const rpca_ctx* c) { return c->h_flags[0]; }
inline int flag_emit_k(const rpca_ctx* c) { return c->h_flags[6]; }
inline int flag_steps_run(const rpca_ctx* c) { return c->h_flags[7]; }
inline int flag_done(const rpca_ctx* c) { return c->h_flags[1]; }
inline int flag_status(const rpca_ctx* c) { return c->h_flags[2]; }
inline int flag_conv(const rpca_ctx* c) { return c->h_flags[3]; }

template <typename T>
int dalloc(T** p, size_t count) {
  if (count == 0) count = 1;
  CK(cudaMalloc((void**)p, count * sizeof(T)));
  return RPCA_OK;
}

}  // namespace

extern "C" {

const char* rpca_status_string(int s) {
  switch (s) {
    case RPCA_OK: return "RPCA_OK";
    case RPCA_ERR_INVALID_ARG: return "RPCA_ERR_INVALID_ARG";
    case RPCA_ERR_CUDA: return "RPCA_ERR_CUDA";
    case RPCA_ERR_NUMERICAL: return "RPCA_ERR_NUMERICAL";
    case RPCA_ERR_CAPACITY: return "RPCA_ERR_CAPACITY";
    case RPCA_ERR_NOT_CONVERGED: return "RPCA_ERR_NOT_CONVERGED";
    case RPCA_ERR_TIMEOUT: return "RPCA_ERR_TIMEOUT";
    case RPCA_ERR_STATE: return "RPCA_ERR_STATE";
  }
  return "RPCA_UNKNOWN_STATUS";
}

int rpca_params_default(rpca_params* p) {
  if (!p) return RPCA_ERR_INVALID_ARG;
  memset(p, 0, sizeof(*p));
  p->max_iter = 100;
  p->trim = 1;
  p->precision = RPCA_PREC_FP32;
  p->zeta_mode = RPCA_ZETA_PAPER;
  return RPCA_OK;
}

// Unique id of the current CUDA context (0 if unavailable): a device reset or a context
// teardown between calls gives a new id, and the cached objects, which belonged to the old
// context, are then dropped without touching them (their memory went with that context).
static unsigned long long current_context_id() {
  using GetCurrent = CUresult (*)(CUcontext*);
  using GetId = CUresult (*)(CUcontext, unsigned long long*);
  static GetCurrent get_current = nullptr;
  static GetId get_id = nullptr;
  if (!get_current || !get_id) {
    cudaDriverEntryPointQueryResult q1, q2;
    if (cudaGetDriverEntryPointByVersion("cuCtxGetCurrent", (void**)&get_current, 12000, cudaEnableDefault, &q1) !=
            cudaSuccess ||
        cudaGetDriverEntryPointByVersion("cuCtxGetId", (void**)&get_id, 12000, cudaEnableDefault, &q2) !=
            cudaSuccess ||
        q1 != cudaDriverEntryPointSuccess || q2 != cudaDriverEntryPointSuccess) {
      get_current = nullptr;
      get_id = nullptr;
      return 0;
    }
  }
  cudaFree(nullptr);  // makes the runtime's context current
  CUcontext cx = nullptr;
  unsigned long long id = 0;
  if (get_current(&cx) != CUDA_SUCCESS || !cx || get_id(cx, &id) != CUDA_SUCCESS) return 0;
  return id;
}

static unsigned long long g_attr_ctx = 0;

int rpca_create(rpca_ctx** out, const rpca_params* params, void* stream) {
  if (!out || !params) return RPCA_ERR_INVALID_ARG;
  *out = nullptr;
  const rpca_params& p = *params;
  if (!(p.beta > 0) || !(p.gamma >= 0 && p.gamma < 1) || !(p.tol >= 0) || p.max_iter < 0 ||
      p.precision < RPCA_PREC_FP64 || p.precision > RPCA_PREC_BF16_SPLIT || p.zeta_mode < 0 || p.zeta_mode > 3 ||
      p.beta_init < 0 || p.mu_trim < 0 || p.pass_kind < 0 || p.pass_kind > 2 || !(p.split_switch >= 0) ||
      p.observed < RPCA_OBS_ALL || p.observed > RPCA_OBS_NAN ||
      (p.observed == RPCA_OBS_NAN && p.zeta_mode == RPCA_ZETA_LEARNED))
    return RPCA_ERR_INVALID_ARG;
  {
    // a context the kernel attributes were not set in (the first, or a new one after a device
    // reset): the launchers set them again
    const unsigned long long cid = current_context_id();
    if (cid != g_attr_ctx) {
      g_attr_ctx = cid;
      ++g_attr_epoch;
    }
  }
  rpca_ctx* c = new (std::nothrow) rpca_ctx();
  if (!c) return RPCA_ERR_CUDA;
  c->p = p;
  if (c->p.init_max_passes <= 0) c->p.init_max_passes = 40;
  c->prec = (p.precision == RPCA_PREC_FP64) ? PREC_F64 : PREC_F32;
  c->dmode = (p.precision == RPCA_PREC_BF16 || p.precision == RPCA_PREC_BF16_SPLIT) ? 1 : 0;
  c->split = p.precision == RPCA_PREC_BF16_SPLIT;
  c->tsize = (c->prec == PREC_F32) ? 4 : 8;
  if (c->p.init_tol <= 0) c->p.init_tol = (c->prec == PREC_F32) ? 1e-5 : 1e-13;
  c->stream = static_cast<cudaStream_t>(stream);
  if (cudaGetDevice(&c->device) != cudaSuccess || cudaMallocHost((void**)&c->h_flags, 8 * sizeof(int)) != cudaSuccess) {
    delete c;
    return RPCA_ERR_CUDA;
  }
  c->small_grid = small_grid_size(c->device);
  *out = c;
  return RPCA_OK;
}

void rpca_destroy(rpca_ctx* c) {
  if (!c) return;
  if (c->stream) cudaStreamSynchronize(c->stream);
  else cudaDeviceSynchronize();
  prof_collect(c, 0);
  for (cudaEvent_t e : c->ev_free) cudaEventDestroy(e);
  free_workspace(c);
  if (c->theta) cudaFree(c->theta);
  if (c->obs_count) cudaFree(c->obs_count);
  if (c->h_flags) cudaFreeHost(c->h_flags);
  delete c;
}

int rpca_init(rpca_ctx* c, const void* D, int64_t m, int64_t n, int64_t ld, int dtype, int r) {
  if (!c || !D || m < 1 || n < 1 || ld < n || r < 1 || r > kMaxR || 2 * (int64_t)r > (m < n ? m : n) ||
      (dtype != RPCA_DTYPE_F32 && dtype != RPCA_DTYPE_F64) || m > (1ll << 30) || n > (1ll << 30) ||
      m * n > (1ll << 40))
    return RPCA_ERR_INVALID_ARG;
  const bool reuse = c->U && c->ws_m == m && c->ws_n == n && c->ws_r == r;
  if (!reuse) free_workspace(c);
  c->ready = false;
  c->m = m;
  c->n = n;
  c->r = r;
  c->Rr = padded_rank(r);
  // block size of the initial subspace iteration: oversample to 8 columns for r <= 6 (the
  // tensor-core pass then runs the initialisation in its rank-8 image layout), else 2r up to 16
  int b = (r <= 6) ? 8 : ((2 * r <= 16) ? 2 * r : 16);
  const int64_t mn_min = m < n ? m : n;
  if (b > mn_min) b = (int)(mn_min & ~1ll);
  if (b < r) b = r + (r & 1);
  c->b = b;
  c->Rb = padded_rank(b);
  if (c->Rr < 0 || c->Rb < 0) return RPCA_ERR_INVALID_ARG;
  const int want = (c->prec == PREC_F32) ? RPCA_DTYPE_F32 : RPCA_DTYPE_F64;
  if (dtype == want) {
    c->D = D;
    c->ld = ld;
  } else {
    if (!c->Down) CK(cudaMalloc(&c->Down, (size_t)m * n * c->tsize));
    if (dtype == RPCA_DTYPE_F64)
      CK(launch_convert_f64_to_f32((const double*)D, ld, (float*)c->Down, (int)m, (int)n, c->stream));
    else
      CK(launch_convert_f32_to_f64((const float*)D, ld, (double*)c->Down, (int)m, (int)n, c->stream));
    c->D = c->Down;
    c->ld = n;
  }
  c->vec = ((reinterpret_cast<uintptr_t>(c->D) & 15) == 0 && ((c->ld * (int64_t)c->tsize) & 15) == 0) ? 1 : 0;
  c->tc_iter = c->tc_init = false;
  if (c->prec == PREC_F32 && (c->vec || c->dmode) && c->p.pass_kind != RPCA_PASS_SIMT) {
    int nsm = 0;
    cudaDeviceGetAttribute(&nsm, cudaDevAttrMultiProcessorCount, c->device);
    c->TR = (int)((m + 127) / 128);
    c->TC = (int)((n + 63) / 64);
    const bool it = tc_pass_supported(c->Rr), in = tc_pass_supported(c->Rb);
    int max_ct = 1 << 30;
    if (it) max_ct = std::min(max_ct, tc_max_col_tiles(c->Rr));
    if (in) max_ct = std::min(max_ct, tc_max_col_tiles(c->Rb));
    if (nsm > 0 && (it || in) && ((reuse && c->plan.ncta > 0) || tc_plan(c->TR, c->TC, nsm, max_ct, &c->plan))) {
      c->tc_iter = it;
      c->tc_init = in;
    }
  }
  if (c->dmode) {
    c->ldb = (n + 7) & ~7ll;  // 16-byte row stride
    const size_t part = (size_t)m * c->ldb * 2;
    if (!c->Dhl) CK(cudaMalloc(&c->Dhl, c->split ? 2 * part : part));
    CK(launch_convert_f32_to_bf16x2(static_cast<const float*>(c->D), c->ld, c->Dhl,
                                    c->split ? static_cast<uint8_t*>(c->Dhl) + part : nullptr, c->ldb, (int)m,
                                    (int)n, c->stream));
  }
  if ((c->tc_iter || c->tc_init) && !encode_dmap(c)) c->tc_iter = c->tc_init = false;

  const int w = c->b > c->r ? c->b : c->r;
  const int Rmax = c->Rb > c->Rr ? c->Rb : c->Rr;
  size_t p1 = 0, p2 = 0, ncta = 0;
  for (int R : {c->Rr, c->Rb}) {
    const PassGeom pg = pass_geometry(c->prec, R);
    const Grid gs{(int)((n + pg.BW - 1) / pg.BW), (int)((m + pg.BH - 1) / pg.BH), 0};
    const Grid gt{c->plan.Bmax, c->plan.S2, c->plan.ncta};
    // partial slices: SIMT pass [n_p][rows][R]; tensor-core pass Y1 [Bmax][m][R] and Y2
    // [S2][n][RK] (rows padded to the image rank)
    p1 = std::max(p1, std::max((size_t)gs.n_p1 * m * R, (size_t)gt.n_p1 * m * R));
    p2 = std::max(p2, std::max((size_t)gs.n_p2 * n * R, (size_t)gt.n_p2 * n * (size_t)tc_image_rank(R)));
    ncta = ncta > (size_t)gs.n_p1 * gs.n_p2 ? ncta : (size_t)gs.n_p1 * gs.n_p2;
    ncta = ncta > (size_t)gt.n_cta ? ncta : (size_t)gt.n_cta;
  }
  int st = RPCA_OK;
  if (!reuse) {
  const size_t ts = c->tsize;
  CK(cudaMalloc(&c->U, (size_t)m * r * ts));
  CK(cudaMalloc(&c->sig, 16 * ts));
  CK(cudaMalloc(&c->V, (size_t)n * r * ts));
  CK(cudaMalloc(&c->Ut, (size_t)m * w * ts));
  CK(cudaMalloc(&c->Vt, (size_t)n * w * ts));
  CK(cudaMalloc(&c->Y1, (size_t)m * w * ts));
  CK(cudaMalloc(&c->Y2, (size_t)n * w * ts));
  CK(cudaMalloc(&c->part, (size_t)c->small_grid * kSmallSlots * 256 * sizeof(double)));
  if ((st = dalloc(&c->resP, ncta)) ||
      (st = dalloc(&c->nnzP, ncta)) || (st = dalloc(&c->st, 1)) || (st = dalloc(&c->stats, (size_t)c->p.max_iter + 2)))
    return st;
  CK(cudaMalloc(&c->Wc, (size_t)m * Rmax * c->tsize));
  CK(cudaMalloc(&c->Utc, (size_t)m * Rmax * c->tsize));
  CK(cudaMalloc(&c->Vc, (size_t)n * Rmax * c->tsize));
  CK(cudaMalloc(&c->Vtc, (size_t)n * Rmax * c->tsize));
  CK(cudaMalloc(&c->P1, p1 * c->tsize));
  CK(cudaMalloc(&c->P2, p2 * c->tsize));
  if (c->TR > 0) {
    if (c->tc_iter || c->tc_init) {
      const int nc = c->plan.ncta;
      CK(cudaMalloc((void**)&c->d_rect, sizeof(int4) * nc));
      CK(cudaMalloc((void**)&c->d_ids, sizeof(int4) * nc));
      CK(cudaMalloc((void**)&c->d_p1nsl, sizeof(int) * c->TR));
      CK(cudaMalloc((void**)&c->tfac, sizeof(float) * 1024));
      if (c->tc_iter && !c->dmode) {
        CK(cudaMalloc((void**)&c->swords, sizeof(unsigned) * (size_t)m * 2 * c->TC));
        CK(cudaMalloc((void**)&c->wcc, sizeof(unsigned) * (size_t)m * ((2 * c->TC + kWordChunk - 1) / kWordChunk)));
      }
      CK(cudaMemcpy(c->d_rect, c->plan.rect.data(), sizeof(int4) * nc, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c->d_ids, c->plan.ids.data(), sizeof(int4) * nc, cudaMemcpyHostToDevice));
      CK(cudaMemcpy(c->d_p1nsl, c->plan.p1_nsl.data(), sizeof(int) * c->TR, cudaMemcpyHostToDevice));
    }
    // zero-filled: rows past m, n are never written and must read as zero
    for (int set = 0; set < 2; ++set) {
      CK(cudaMalloc((void**)&c->wop[set], (size_t)c->TR * img::WOP_MAX));
      CK(cudaMalloc((void**)&c->utop[set], (size_t)c->TR * img::UTOP_MAX));
      CK(cudaMalloc((void**)&c->vop[set], (size_t)c->TC * img::VOP_MAX));
      CK(cudaMalloc((void**)&c->vtop[set], (size_t)c->TC * img::VTOP_MAX));
      CK(cudaMemsetAsync(c->wop[set], 0, (size_t)c->TR * img::WOP_MAX, c->stream));
      CK(cudaMemsetAsync(c->utop[set], 0, (size_t)c->TR * img::UTOP_MAX, c->stream));
      CK(cudaMemsetAsync(c->vop[set], 0, (size_t)c->TC * img::VOP_MAX, c->stream));
      CK(cudaMemsetAsync(c->vtop[set], 0, (size_t)c->TC * img::VTOP_MAX, c->stream));
    }
  }
  if (learned(c)) {
    // SIMT pass: rows of VW words per sub-chunk of 32 VW columns (VW = 4 in FP32, 2 in FP64);
    // tensor-core pass: 256 words per 128 x 64 tile, tile-major
    const long long wr_simt = (c->prec == PREC_F32) ? 4 * ((n + 127) / 128) : 2 * ((n + 63) / 64);
    c->mask_wr = wr_simt;
    c->mask_words = std::max(wr_simt * m, 256ll * ((m + 127) / 128) * ((n + 63) / 64));
    CK(cudaMalloc((void**)&c->masks, sizeof(unsigned) * 2 * (size_t)c->mask_words));
    CK(cudaMemsetAsync(c->masks, 0, sizeof(unsigned) * 2 * (size_t)c->mask_words, c->stream));
    if ((st = dalloc(&c->chgP, ncta))) return st;
  }
  c->ws_m = m;
  c->ws_n = n;
  c->ws_r = r;
  }
  CK(cudaMemsetAsync(c->stats, 0, sizeof(DevStats) * ((size_t)c->p.max_iter + 2), c->stream));
  CK(cudaMemsetAsync(c->sig, 0, 16 * c->tsize, c->stream));
  // partial observation: p = |observed entries| / (m n)
  double inv_p = 1.0;
  if (c->p.observed == RPCA_OBS_NAN) {
    if (!c->obs_count) CK(cudaMalloc((void**)&c->obs_count, sizeof(unsigned long long)));
    unsigned long long cnt = 0;
    CK(launch_count_observed(c->D, c->ld, (int)m, (int)n, c->prec == PREC_F32, c->obs_count, c->stream));
    CK(cudaMemcpyAsync(&cnt, c->obs_count, sizeof(cnt), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (cnt == 0) return RPCA_ERR_INVALID_ARG;
    inv_p = (double)m * (double)n / (double)cnt;
  }

  DevState h;
  memset(&h, 0, sizeof(h));
  const double root = sqrt((double)m * (double)n);
  h.beta = c->p.beta;
  h.gamma = c->p.gamma;
  h.tol = c->p.tol;
  h.beta_init = c->p.beta_init > 0 ? c->p.beta_init : 2.0 * c->p.beta;
  h.mu_trim = c->p.mu_trim > 0 ? c->p.mu_trim : 2.0 * c->p.beta * root / r;
  h.max_iter = c->p.max_iter;
  h.zeta_mode = c->p.zeta_mode;
  h.trim = c->p.trim;
  h.zeta = INFINITY;
  h.split_switch = c->split ? (c->p.split_switch > 0 ? c->p.split_switch : 1e-2) : 0.0;
  h.inv_p = inv_p;
  h.emit_k = -1;
  CK(cudaMemcpyAsync(c->st, &h, sizeof(h), cudaMemcpyHostToDevice, c->stream));
  c->h_flags[7] = 0;  // steps_run as uploaded

  // Algorithm 3.  Phase A: sigma_1(D) with L = 0 and no threshold; phase B: top-r SVD of
  // D - S_{-1} (the pass with L = 0 and zeta_{-1} keeps exactly D_ij where |D_ij| <= zeta).
  // The phase and step counters live in DevState; steps are queued in batches and the ones
  // behind the final convergence return at once (DevState.done), so the host waits once per
  // batch.  Each phase accepts its step init_max_passes - 1 as converged, so 2 init_max_passes
  // steps always finish.
  prof_break(c);
  SmallArgs ra = small_args(c, SM_RAND, c->Rb);
  if ((st = run_small(c, ra))) return st;
  const int cap = 2 * c->p.init_max_passes;
  bool conv = false;
  for (int steps = 0; steps < cap && !conv;) {
    // each phase takes two steps at least (its first step is never accepted unless it is
    // the last allowed one); the first batch has five steps (most initialisations end there),
    // later ones two (a step queued behind the convergence costs a few microseconds, a wait
    // for the host more)
    int batch = (steps == 0) ? 5 : 2;
    if (batch > cap - steps) batch = cap - steps;
    for (int i = 0; i < batch; ++i) {
      if ((st = run_pass(c, c->Rb, true))) return st;
      if ((st = run_small(c, small_args(c, SM_RR, c->Rb)))) return st;
    }
    steps += batch;
    const int run0 = flag_steps_run(c);
    if ((st = read_flags(c))) return st;
    prof_collect(c, flag_steps_run(c) - run0);  // the passes queued behind convergence did no work
    if (flag_status(c)) return flag_status(c);
    conv = flag_conv(c) != 0;
  }
  if (!conv) return RPCA_ERR_NOT_CONVERGED;  // not reached: the last step of each phase is accepted
  CK(cudaMemsetAsync(&c->st->done, 0, sizeof(int), c->stream));
  c->h_flags[1] = 0;  // done, as just reset (the other flags were read after the last step)
  c->ready = true;
  return RPCA_OK;
}

int rpca_get_pass_kind(rpca_ctx* c, int* iteration_kind, int* init_kind) {
  if (!c) return RPCA_ERR_INVALID_ARG;
  if (!c->ready) return RPCA_ERR_STATE;
  if (iteration_kind) *iteration_kind = c->tc_iter ? RPCA_PASS_TENSOR : RPCA_PASS_SIMT;
  if (init_kind) *init_kind = c->tc_init ? RPCA_PASS_TENSOR : RPCA_PASS_SIMT;
  return RPCA_OK;
}

int rpca_set_zeta(rpca_ctx* c, double zeta) {
  if (!c || !c->ready || !(zeta >= 0)) return RPCA_ERR_INVALID_ARG;
  CK(cudaMemcpyAsync(&c->st->zeta, &zeta, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  // the support words, if any, were taken with the former threshold
  const int none = -1;
  CK(cudaMemcpyAsync(&c->st->emit_k, &none, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  c->h_flags[6] = -1;
  return RPCA_OK;
}

int rpca_iterate(rpca_ctx* c, int n_iters, rpca_iter_stats* out, int* n_done) {
  if (n_done) *n_done = 0;
  if (!c || n_iters < 0) return RPCA_ERR_INVALID_ARG;
  if (!c->ready || (learned(c) && !c->theta_set)) return RPCA_ERR_STATE;
  int st;
  // the host's copy of the state flags is current (every call that changes them on the device
  // reads them back or sets them), so the first chunk goes out without a wait
  const int k0 = flag_k(c);
  int done = flag_done(c);
  int launched = 0;
  const int max_stats = c->p.max_iter + 2 - k0;  // DevStats entries from k0 on
  std::vector<DevStats> hs;
  while (!done && launched < n_iters) {
    // the first chunk as long as the last solve on this context took (at least 8), later ones
    // 4; the passes queued behind convergence return at once
    const int want = launched == 0 ? std::min(32, std::max(8, c->last_iters + 1)) : 4;
    const int chunk = std::min(n_iters - launched, want);
    for (int i = 0; i < chunk; ++i) {
      if ((st = run_pass(c, c->Rr, false))) return st;
      if ((st = run_small(c, small_args(c, SM_UPDATE, c->Rr)))) return st;
    }
    launched += chunk;
    // the flags and the statistics of every pass launched so far, in one wait
    const int ns = std::min(max_stats, launched + 1);
    hs.resize((size_t)std::max(ns, 1));
    prof_break(c);
    CK(cudaMemcpyAsync(c->h_flags, &c->st->k, 8 * sizeof(int), cudaMemcpyDeviceToHost, c->stream));
    if (ns > 0) CK(cudaMemcpyAsync(hs.data(), c->stats + k0, sizeof(DevStats) * ns, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    if (flag_status(c)) return flag_status(c);
    done = flag_done(c);
  }
  const int k1 = flag_k(c);
  int count = k1 - k0 + (flag_done(c) ? 1 : 0);
  if (count > n_iters) count = n_iters;
  if (count < 0) count = 0;
  prof_collect(c, count);
  const int need = std::max(count, flag_done(c) ? k1 - k0 + 1 : 0);
  if ((int)hs.size() < need) {  // no chunk ran (already done): the statistics held
    hs.resize((size_t)need);
    CK(cudaMemcpyAsync(hs.data(), c->stats + k0, sizeof(DevStats) * need, cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
  }
  if (out)
    for (int i = 0; i < count; ++i) {
      out[i].k = hs[i].k;
      out[i].err = hs[i].err;
      out[i].zeta = hs[i].zeta;
      out[i].sigma1 = hs[i].sigma1;
      out[i].sigma_r1 = hs[i].sigma_r1;
      out[i].nnz = hs[i].nnz;
      out[i].zeta_next_plain = hs[i].zeta_next_plain;
      out[i].g = hs[i].g;
      for (int f = 0; f < 6; ++f) out[i].features[f] = hs[i].feat[f];
      out[i].support_changes = hs[i].changes;
    }
  if (n_done) *n_done = count;
  if (flag_done(c)) {
    const DevStats& last = hs[(size_t)(k1 - k0)];
    c->last_nnz = last.nnz;  // the support the pass at iterate k1 counted
    c->last_nnz_k = k1;
    c->last_iters = k1;
    return (last.err < c->p.tol) ? RPCA_OK : RPCA_ERR_NOT_CONVERGED;
  }
  return RPCA_ERR_NOT_CONVERGED;
}

int rpca_set_schedule(rpca_ctx* c, const float* theta, int depth) {
  if (!c || !theta || depth < 1) return RPCA_ERR_INVALID_ARG;
  if (!learned(c)) return RPCA_ERR_STATE;
  if (!c->theta) CK(cudaMalloc((void**)&c->theta, sizeof(float) * mlp::NPARAM));
  CK(cudaMemcpyAsync(c->theta, theta, sizeof(float) * mlp::NPARAM, cudaMemcpyDeviceToDevice, c->stream));
  c->depth = depth;
  c->theta_set = true;
  return RPCA_OK;
}

int rpca_get_pass_operands(rpca_ctx* c, void* W, void* V, void* Ut, void* Vt, int* width) {
  if (!c || !W || !V || !Ut || !Vt || !width) return RPCA_ERR_INVALID_ARG;
  if (!c->ready) return RPCA_ERR_STATE;
  *width = c->Rr;
  const size_t rm = (size_t)c->m * c->Rr * c->tsize, rn = (size_t)c->n * c->Rr * c->tsize;
  CK(cudaMemcpyAsync(W, c->Wc, rm, cudaMemcpyDeviceToDevice, c->stream));
  CK(cudaMemcpyAsync(V, c->Vc, rn, cudaMemcpyDeviceToDevice, c->stream));
  // the pass reads the trimmed factors; their orthonormal bases come from a small kernel
  CK(cudaMemsetAsync(Ut, 0, rm, c->stream));
  CK(cudaMemsetAsync(Vt, 0, rn, c->stream));
  SmallArgs b = small_args(c, SM_BASES, c->Rr);
  b.out_ut = Ut;
  b.out_vt = Vt;
  return run_small(c, b);
}

int rpca_get_lowrank(rpca_ctx* c, double* U, double* sigma, double* V) {
  if (!c || !U || !sigma || !V) return RPCA_ERR_INVALID_ARG;
  if (!c->ready) return RPCA_ERR_STATE;
  if (c->prec == PREC_F64) {
    CK(cudaMemcpyAsync(U, c->U, sizeof(double) * c->m * c->r, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(sigma, c->sig, sizeof(double) * c->r, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(V, c->V, sizeof(double) * c->n * c->r, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    CK(launch_convert_f32_to_f64(static_cast<const float*>(c->U), c->r, U, (int)c->m, c->r, c->stream));
    CK(launch_convert_f32_to_f64(static_cast<const float*>(c->sig), c->r, sigma, 1, c->r, c->stream));
    CK(launch_convert_f32_to_f64(static_cast<const float*>(c->V), c->r, V, (int)c->n, c->r, c->stream));
  }
  return RPCA_OK;
}

int rpca_get_state(rpca_ctx* c, int* k, double* zeta, int* flags) {
  if (!c || !k || !zeta) return RPCA_ERR_INVALID_ARG;
  if (!c->ready) return RPCA_ERR_STATE;
  int use_lo = 0;
  CK(cudaMemcpyAsync(k, &c->st->k, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(zeta, &c->st->zeta, sizeof(double), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaMemcpyAsync(&use_lo, &c->st->use_lo, sizeof(int), cudaMemcpyDeviceToHost, c->stream));
  CK(cudaStreamSynchronize(c->stream));
  if (flags) *flags = use_lo ? RPCA_STATE_READS_LO : 0;
  return RPCA_OK;
}

int rpca_set_lowrank(rpca_ctx* c, const double* U, const double* sigma, const double* V, int k, double zeta,
                     int flags) {
  if (!c || !U || !sigma || !V || k < 0 || !(zeta >= 0) || (flags & ~RPCA_STATE_READS_LO)) return RPCA_ERR_INVALID_ARG;
  if (!c->ready) return RPCA_ERR_STATE;
  if (k > c->p.max_iter) return RPCA_ERR_INVALID_ARG;
  if (c->prec == PREC_F64) {
    CK(cudaMemcpyAsync(c->U, U, sizeof(double) * c->m * c->r, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->sig, sigma, sizeof(double) * c->r, cudaMemcpyDeviceToDevice, c->stream));
    CK(cudaMemcpyAsync(c->V, V, sizeof(double) * c->n * c->r, cudaMemcpyDeviceToDevice, c->stream));
  } else {
    CK(launch_convert_f64_to_f32(U, c->r, static_cast<float*>(c->U), (int)c->m, c->r, c->stream));
    CK(launch_convert_f64_to_f32(sigma, c->r, static_cast<float*>(c->sig), 1, c->r, c->stream));
    CK(launch_convert_f64_to_f32(V, c->r, static_cast<float*>(c->V), (int)c->n, c->r, c->stream));
  }
  // iteration state: L_k held, zeta_k for the next pass, running again; a BF16_SPLIT solve
  // that had switched to hi + lo keeps reading it
  const int zero = 0;
  const int use_lo = (c->split && (flags & RPCA_STATE_READS_LO)) ? 1 : 0;
  CK(cudaMemcpyAsync(&c->st->k, &k, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(&c->st->zeta, &zeta, sizeof(double), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(&c->st->done, &zero, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  CK(cudaMemcpyAsync(&c->st->use_lo, &use_lo, sizeof(int), cudaMemcpyHostToDevice, c->stream));
  const int no_emit[2] = {0, -1};  // emit, emit_k: no support words for this iterate yet
  CK(cudaMemcpyAsync(&c->st->emit, no_emit, sizeof(no_emit), cudaMemcpyHostToDevice, c->stream));
  // Trim (Algorithm 2), orthonormal bases and the copies (and images) read by the next pass
  int st = run_small(c, small_args(c, SM_PREPARE, c->Rr));
  if (st) return st;
  if ((st = read_flags(c))) return st;
  prof_collect(c, 0);
  return flag_status(c);
}

int rpca_selftest_waits(int* mbar_status, int* grid_status) {
  if (!mbar_status || !grid_status) return RPCA_ERR_INVALID_ARG;
  return run_wait_selftest(mbar_status, grid_status) == cudaSuccess ? RPCA_OK : RPCA_ERR_CUDA;
}

int rpca_get_sparse(rpca_ctx* c, int64_t* idx, double* val, int64_t cap, int64_t* nnz) {
  if (!c || !nnz || cap < 0 || (cap > 0 && (!idx || !val))) return RPCA_ERR_INVALID_ARG;
  if (!c->ready) return RPCA_ERR_STATE;
  if (!c->rowcnt) {
    CK(cudaMalloc((void**)&c->rowcnt, sizeof(unsigned long long) * c->m));
    CK(cudaMalloc((void**)&c->rowoff, sizeof(unsigned long long) * (c->m + 1)));
  }
  ExtractArgs a;
  memset(&a, 0, sizeof(a));
  a.D = c->D;
  a.ld = c->ld;
  a.m = (int)c->m;
  a.n = (int)c->n;
  a.W = c->Wc;
  a.V = c->Vc;
  a.st = c->st;
  a.rowcnt = c->rowcnt;
  a.rowoff = c->rowoff;
  a.idx = (long long*)idx;
  a.val = val;
  a.vec = c->vec;
  // S_k from the support words when the last pass wrote them for the iterate held
  // (FP32 D, tensor-core pass; the host's copy of the state flags is current after
  // rpca_iterate, rpca_init and rpca_set_lowrank): their count is the one that pass reported,
  // so no count has to come back first.  Otherwise two passes over D.
  const bool from_words = c->swords != nullptr && flag_emit_k(c) == flag_k(c) && c->last_nnz_k == flag_k(c);
  unsigned long long total = 0;
  if (from_words) {
    total = (unsigned long long)c->last_nnz;
    *nnz = (int64_t)total;
    if ((int64_t)total > cap) return RPCA_ERR_CAPACITY;
    prof_break(c);
    prof_mark(c, false, true);
    CK(cudaMemsetAsync(c->rowcnt, 0, sizeof(unsigned long long) * c->m, c->stream));
    CK(launch_words_count(c->swords, 2 * c->TC, (int)c->m, c->wcc, c->rowcnt, c->stream));
    prof_mark(c, false, false);
    prof_mark(c, false, true);
    CK(launch_scan_rows(c->rowcnt, c->rowoff, (int)c->m, c->stream));
    prof_mark(c, false, false);
    prof_mark(c, false, true);
    if (total > 0) CK(launch_extract_words_f32(c->Rr, a, c->swords, c->wcc, 2 * c->TC, c->stream));
    prof_mark(c, false, false);
    // the count was known: return with the writes queued on the stream (their profile spans
    // are collected at the next wait)
    prof_break(c);
    return RPCA_OK;
  } else {
    prof_break(c);
    prof_mark(c, false, true);
    CK(launch_extract_count(c->prec, c->Rr, a, c->stream));
    prof_mark(c, false, false);
    prof_mark(c, false, true);
    CK(launch_scan_rows(c->rowcnt, c->rowoff, (int)c->m, c->stream));
    prof_mark(c, false, false);
    CK(cudaMemcpyAsync(&total, c->rowoff + c->m, sizeof(total), cudaMemcpyDeviceToHost, c->stream));
    CK(cudaStreamSynchronize(c->stream));
    *nnz = (int64_t)total;
    prof_break(c);
    if ((int64_t)total > cap) {
      prof_collect(c, 0);
      return RPCA_ERR_CAPACITY;
    }
    prof_mark(c, false, true);
    CK(launch_extract_write(c->prec, c->Rr, a, c->stream));
    prof_mark(c, false, false);
  }
  CK(cudaStreamSynchronize(c->stream));
  prof_collect(c, 0);
  return RPCA_OK;
}

int rpca_set_profiling(rpca_ctx* c, int on) {
  if (!c) return RPCA_ERR_INVALID_ARG;
  CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
  if (on < 0) return RPCA_ERR_INVALID_ARG;
  prof_collect(c, 0);
  c->prof = on != 0;
  c->prof_stride = on > 1 ? on : 1;
  c->pass_seq = 0;
  c->pass_ms = c->other_ms = 0;
  c->pass_n = c->other_n = 0;
  return RPCA_OK;
}

int rpca_get_profile(rpca_ctx* c, double* pass_ms, int64_t* pass_launches, double* other_ms,
                     int64_t* other_launches) {
  if (!c) return RPCA_ERR_INVALID_ARG;
  CK(c->stream ? cudaStreamSynchronize(c->stream) : cudaDeviceSynchronize());
  prof_collect(c, 0);
  if (pass_ms) *pass_ms = c->pass_ms;
  if (pass_launches) *pass_launches = c->pass_n;
  if (other_ms) *other_ms = c->other_ms;
  if (other_launches) *other_launches = c->other_n;
  return RPCA_OK;
}

// init + iterate to tolerance + outputs on context c (parameters beta, gamma, tol set here).
static int solve_on(rpca_ctx* c, const float* D, int64_t m, int64_t n, int r, double beta, double gamma, double tol,
                    double* U, double* sigma, double* V, int64_t* s_idx, double* s_val, int64_t s_cap, int64_t* nnz,
                    int* iters, double* err) {
  c->p.beta = beta;
  c->p.gamma = gamma;
  c->p.tol = tol;
  int result = rpca_init(c, D, m, n, n, RPCA_DTYPE_F32, r);
  if (!result) {
    std::vector<rpca_iter_stats> hs((size_t)c->p.max_iter + 1);
    int done = 0;
    result = rpca_iterate(c, c->p.max_iter + 1, hs.data(), &done);
    if (iters) *iters = done > 0 ? hs[done - 1].k : 0;
    if (err) *err = done > 0 ? hs[done - 1].err : NAN;
    if (result == RPCA_OK || result == RPCA_ERR_NOT_CONVERGED) {
      int s2 = rpca_get_lowrank(c, U, sigma, V);
      if (!s2) s2 = rpca_get_sparse(c, s_idx, s_val, s_cap, nnz);
      if (s2) result = s2;
    }
  }
  return result;
}

static int solve_device(const float* D, int64_t m, int64_t n, int r, double beta, double gamma, double tol,
                        double* U, double* sigma, double* V, int64_t* s_idx, double* s_val, int64_t s_cap,
                        int64_t* nnz, int* iters, double* err, cudaStream_t stream) {
  rpca_params p;
  rpca_params_default(&p);
  p.beta = beta;
  p.gamma = gamma;
  p.tol = tol;
  rpca_ctx* c = nullptr;
  int st = rpca_create(&c, &p, stream);
  if (st) return st;
  const int result = solve_on(c, D, m, n, r, beta, gamma, tol, U, sigma, V, s_idx, s_val, s_cap, nnz, iters, err);
  rpca_destroy(c);
  return result;
}

// Device buffers, stream and context of rpca_solve_host, kept between calls (grown as
// needed) so that repeated calls pay for the copies and the solve, not for allocation.
// Serialised by a mutex; freed by rpca_solve_host_release (or with the process).
struct HostSolveCache {
  int device = -1;
  unsigned long long ctx_id = 0;  // CUDA context the cached objects belong to
  size_t d_elems = 0, u_elems = 0, v_elems = 0, cap = 0;
  float* dD = nullptr;
  double *dU = nullptr, *dS = nullptr, *dV = nullptr, *dval = nullptr;
  int64_t* didx = nullptr;
  cudaStream_t s = nullptr;
  rpca_ctx* ctx = nullptr;
};
static std::mutex g_host_mu;
static HostSolveCache* g_host = nullptr;  // heap object: no destructor runs at process exit

static void host_cache_free(HostSolveCache* h) {
  if (!h || h->device < 0) return;
  int cur = 0;
  cudaGetDevice(&cur);
  if (cur != h->device) cudaSetDevice(h->device);
  if (h->s) cudaStreamSynchronize(h->s);
  if (h->ctx) rpca_destroy(h->ctx);
  void* ptrs[] = {h->dD, h->dU, h->dS, h->dV, h->dval, h->didx};
  for (void* q : ptrs)
    if (q) cudaFree(q);
  if (h->s) cudaStreamDestroy(h->s);
  if (cur != h->device) cudaSetDevice(cur);
  *h = HostSolveCache();
}

// Host-side release of a context whose CUDA objects no longer exist (no CUDA call).
static void forget_ctx(rpca_ctx* c) {
  if (!c) return;
  c->ev_free.clear();
  c->ev_line.clear();
  delete c;
}

// Grows a cached device array to at least `need` elements of `size` bytes.
static bool grow(void** p, size_t* have, size_t need, size_t size) {
  if (*p && *have >= need) return true;
  if (*p) cudaFree(*p);
  *p = nullptr;
  *have = 0;
  if (cudaMalloc(p, need * size) != cudaSuccess) return false;
  *have = need;
  return true;
}

int rpca_solve(const float* D, int64_t m, int64_t n, int r, double beta, double gamma, double tol, double* U,
               double* sigma, double* V, int64_t* s_idx, double* s_val, int64_t s_cap, int64_t* nnz, int* iters,
               double* err) {
  if (!D || !U || !sigma || !V || !nnz) return RPCA_ERR_INVALID_ARG;
  return solve_device(D, m, n, r, beta, gamma, tol, U, sigma, V, s_idx, s_val, s_cap, nnz, iters, err, nullptr);
}

int rpca_solve_host(const float* D, int64_t m, int64_t n, int r, double beta, double gamma, double tol, double* U,
                    double* sigma, double* V, int64_t* s_idx, double* s_val, int64_t s_cap, int64_t* nnz, int* iters,
                    double* err) {
  if (!D || !U || !sigma || !V || !nnz || m < 1 || n < 1 || r < 1 || r > kMaxR || s_cap < 0 ||
      (s_cap > 0 && (!s_idx || !s_val)))
    return RPCA_ERR_INVALID_ARG;
  std::lock_guard<std::mutex> lock(g_host_mu);
  int dev = 0;
  if (cudaGetDevice(&dev) != cudaSuccess) return RPCA_ERR_CUDA;
  if (!g_host) g_host = new (std::nothrow) HostSolveCache();
  if (!g_host) return RPCA_ERR_CUDA;
  HostSolveCache& h = *g_host;
  const unsigned long long cid = current_context_id();
  if (h.device == dev && h.ctx_id != cid) {
    // the context changed under the cache (device reset, context teardown): its objects died
    // with the old context, so they are forgotten, not freed
    forget_ctx(h.ctx);
    h = HostSolveCache();
  }
  if (h.device != dev) {
    host_cache_free(&h);
    h.device = dev;
  }
  h.ctx_id = cid;
  if (!h.s && cudaStreamCreateWithFlags(&h.s, cudaStreamNonBlocking) != cudaSuccess) {
    host_cache_free(&h);
    return RPCA_ERR_CUDA;
  }
  if (!h.ctx) {
    rpca_params p;
    rpca_params_default(&p);
    p.beta = beta;
    p.gamma = gamma;
    p.tol = tol;
    if (rpca_create(&h.ctx, &p, h.s) != RPCA_OK) {
      h.ctx = nullptr;
      host_cache_free(&h);
      return RPCA_ERR_CUDA;
    }
  }
  size_t s_have = h.cap, i_have = h.cap;
  const size_t cap = s_cap > 0 ? (size_t)s_cap : 1;
  size_t sig_have = h.dS ? kMaxR : 0;
  if (!grow((void**)&h.dD, &h.d_elems, (size_t)m * n, sizeof(float)) ||
      !grow((void**)&h.dU, &h.u_elems, (size_t)m * r, sizeof(double)) ||
      !grow((void**)&h.dV, &h.v_elems, (size_t)n * r, sizeof(double)) ||
      !grow((void**)&h.dS, &sig_have, kMaxR, sizeof(double)) || !grow((void**)&h.didx, &i_have, cap, sizeof(int64_t)) ||
      !grow((void**)&h.dval, &s_have, cap, sizeof(double))) {
    host_cache_free(&h);
    return RPCA_ERR_CUDA;
  }
  h.cap = std::min(i_have, s_have);
  int result = RPCA_OK;
  if (cudaMemcpyAsync(h.dD, D, sizeof(float) * m * n, cudaMemcpyHostToDevice, h.s) != cudaSuccess) {
    result = RPCA_ERR_CUDA;
  } else {
    result = solve_on(h.ctx, h.dD, m, n, r, beta, gamma, tol, h.dU, h.dS, h.dV, s_cap > 0 ? h.didx : nullptr,
                      s_cap > 0 ? h.dval : nullptr, s_cap, nnz, iters, err);
    if (result == RPCA_OK || result == RPCA_ERR_NOT_CONVERGED) {
      const int64_t nz = (*nnz < s_cap) ? *nnz : s_cap;
      if (cudaMemcpyAsync(U, h.dU, sizeof(double) * m * r, cudaMemcpyDeviceToHost, h.s) ||
          cudaMemcpyAsync(sigma, h.dS, sizeof(double) * r, cudaMemcpyDeviceToHost, h.s) ||
          cudaMemcpyAsync(V, h.dV, sizeof(double) * n * r, cudaMemcpyDeviceToHost, h.s) ||
          (nz > 0 && cudaMemcpyAsync(s_idx, h.didx, sizeof(int64_t) * nz, cudaMemcpyDeviceToHost, h.s)) ||
          (nz > 0 && cudaMemcpyAsync(s_val, h.dval, sizeof(double) * nz, cudaMemcpyDeviceToHost, h.s)) ||
          cudaStreamSynchronize(h.s))
        result = RPCA_ERR_CUDA;
    }
  }
  if (cudaStreamSynchronize(h.s) != cudaSuccess) result = RPCA_ERR_CUDA;
  if (result == RPCA_ERR_CUDA) host_cache_free(&h);  // start from scratch after a CUDA error
  return result;
}

void rpca_solve_host_release(void) {
  std::lock_guard<std::mutex> lock(g_host_mu);
  if (g_host) host_cache_free(g_host);
}

}  // extern "C"
