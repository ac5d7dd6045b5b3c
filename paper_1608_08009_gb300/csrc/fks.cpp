// Fast Kinetic Scheme in one space dimension (boltz_fks_* in include/boltz.h).
//
// Sec. 3.1 of arxiv 1608.08009: each velocity's piecewise-constant distribution is
// transported exactly (Eq. transport, Eq. f_bar), sampled at the cell centres and then
// relaxed there by the collision step (Eq. relax, Eq. f_coll, with the rescaled operator
// Q / tau of the numerical tests); by Eq. expdt the collision's update belongs to the
// interval that covers the centre, so the centre values are all the state there is.
//
// On a uniform mesh the intervals of one x-velocity v_x move together: after a time t
// the centre of cell j lies in the interval that started as cell j - shift(v_x, t), with
// shift = ceil(v_x t / dx - 1/2) (half-open intervals [i dx + s, (i + 1) dx + s), s = v_x t).
// A step from t to t + dt therefore moves each x-velocity's column of centre values by
// d = shift(t + dt) - shift(t) cells, |d| <= 1 under the transport condition
// dt |v_x| <= dx (Eq. Time); cells left uncovered take the state beyond the row's end.
// That move is fused into the collision kernel's loads (CollideArgs::tr), so one launch per
// step reads f once and writes the new f once, out of place.  The host keeps the time t
// (t += dt per step, float64) and passes the shifts as two bit masks over the x-indices.
#include <cmath>
#include <new>
#include <string>

#include "internal.h"

struct boltz_fks_s {
  boltz_grid_s* grid = nullptr;
  int64_t nx = 0;
  double dx = 0.0;
  double t = 0.0;
};

namespace {

// Index shift of the interval covering a cell centre after the intervals moved by v_x t.
int64_t shift_of(double vx, double t, double dx) { return (int64_t)std::ceil(vx * t / dx - 0.5); }

}  // namespace

extern "C" {

boltz_status boltz_fks_create(boltz_grid g, int64_t n_x, double dx, boltz_fks* out) {
  if (!g || !out || n_x < 1 || !(dx > 0) || !(dx < 1e300)) {
    boltz::set_error("bad FKS arguments (grid, n_x >= 1, dx > 0 and finite, out)");
    return BOLTZ_EINVAL;
  }
  if (g->N > 64) {
    boltz::set_error("the transport masks hold at most 64 x-velocities");
    return BOLTZ_EUNSUPPORTED;
  }
  boltz_fks_s* s = new (std::nothrow) boltz_fks_s();
  if (!s) {
    boltz::set_error("out of host memory");
    return BOLTZ_ENOMEM;
  }
  s->grid = g;
  s->nx = n_x;
  s->dx = dx;
  *out = s;
  return BOLTZ_OK;
}

boltz_status boltz_fks_destroy(boltz_fks s) {
  delete s;
  return BOLTZ_OK;
}

boltz_status boltz_fks_time(boltz_fks s, double* t) {
  if (!s || !t) {
    boltz::set_error("null FKS state or output");
    return BOLTZ_EINVAL;
  }
  *t = s->t;
  return BOLTZ_OK;
}

boltz_status boltz_fks_set_time(boltz_fks s, double t) {
  if (!s || !(t >= 0) || !(t < 1e300)) {
    boltz::set_error("null FKS state or time not finite and >= 0");
    return BOLTZ_EINVAL;
  }
  s->t = t;
  return BOLTZ_OK;
}

boltz_status boltz_fks_shifts(boltz_fks s, double dt, int* d) {
  if (!s || !d || !(dt > 0) || !(dt < 1e300)) {
    boltz::set_error("bad FKS shift arguments");
    return BOLTZ_EINVAL;
  }
  const boltz_grid_s* g = s->grid;
  for (int kx = 0; kx < g->N; ++kx) {
    const double vx = -g->L + kx * g->dv;
    d[kx] = (int)(shift_of(vx, s->t + dt, s->dx) - shift_of(vx, s->t, s->dx));
  }
  return BOLTZ_OK;
}

boltz_status boltz_fks_step(boltz_fks s, const boltz_batch* b, const void* f_in, void* f_out, const void* inflow_lo,
                            const void* inflow_hi, double dt, double tau, void* stream) {
  if (!s) {
    boltz::set_error("null FKS state");
    return BOLTZ_EINVAL;
  }
  boltz_status st = boltz::check_batch(b);
  if (st != BOLTZ_OK) return st;
  if (b->grid != s->grid) {
    boltz::set_error("the batch's grid is not the FKS state's grid");
    return BOLTZ_EINVAL;
  }
  if (b->n_cells % s->nx != 0) {
    boltz::set_error("n_cells must be a whole number of rows of n_x cells");
    return BOLTZ_EINVAL;
  }
  if (!(dt > 0) || !(dt < 1e300) || !(tau > 0) || !(tau < 1e300)) {
    boltz::set_error("dt and tau must be positive and finite");
    return BOLTZ_EINVAL;
  }
  const boltz_grid_s* g = s->grid;
  uint64_t pos = 0, neg = 0;
  for (int kx = 0; kx < g->N; ++kx) {
    const double vx = -g->L + kx * g->dv;
    const int64_t d = shift_of(vx, s->t + dt, s->dx) - shift_of(vx, s->t, s->dx);
    if (d > 1 || d < -1) {
      boltz::set_error("dt |v_x| exceeds dx (the transport condition of Eq. Time): a column would move "
                       "by more than one cell");
      return BOLTZ_EINVAL;
    }
    if (d == 1) pos |= 1ull << kx;
    if (d == -1) neg |= 1ull << kx;
  }
  if (b->n_cells > 0) {
    if (!f_in || !f_out || !inflow_lo || !inflow_hi) {
      boltz::set_error("null f_in, f_out or boundary state");
      return BOLTZ_EINVAL;
    }
    if (f_in == f_out) {
      boltz::set_error("the FKS step is out of place: f_out must not be f_in");
      return BOLTZ_EINVAL;
    }
    if ((st = boltz::check_device(g)) != BOLTZ_OK) return st;
    boltz::TransportArgs tr{s->nx, pos, neg, inflow_lo, inflow_hi};
    // forward Euler on the collision stage, projected onto the moments of the
    // transported values (computed by the launch from what it loads)
    st = boltz::launch_collide(g, b->n_cells, b->prec, b->f_is_fp64, f_in, nullptr, f_out, 0.0, 1.0, dt / tau, nullptr,
                               1, 1, (cudaStream_t)stream, nullptr, 0, -1, 0, nullptr, nullptr, &tr);
    if (st != BOLTZ_OK) return st;
  }
  s->t += dt;
  return BOLTZ_OK;
}

}  // extern "C"
