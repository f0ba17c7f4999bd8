// Host build of the double-single helpers of the complex128 fused pass
// (paper_quant_ph_0201042_gb300/csrc/qs_ds.cuh), exported with C linkage
// for tests/test_ds_host.py.  Compiled with -ffp-contract=off so that every
// line of the helpers rounds once, as on the device.
#include "qs_ds.cuh"

using namespace qs::ds;

extern "C" {
void shim_split(double d, float *h, float *l) { split(d, *h, *l); }
double shim_join(float h, float l) { return join(h, l); }
// out = a*x + b*y (complex double-single); each argument 4 floats (rh, rl, ih, il)
void shim_cmad2(const float *a, const float *x, const float *b, const float *y, float *out) {
    const ccst A = {a[0], a[1], a[2], a[3]}, B = {b[0], b[1], b[2], b[3]};
    const camp X = {x[0], x[1], x[2], x[3]}, Y = {y[0], y[1], y[2], y[3]};
    const camp o = cmad2(A, X, B, Y);
    out[0] = o.rh; out[1] = o.rl; out[2] = o.ih; out[3] = o.il;
}
// out = a*x + b*y with real a, b (only a[0..1], b[0..1] are read)
void shim_rmad2(const float *a, const float *x, const float *b, const float *y, float *out) {
    const ccst A = {a[0], a[1], a[2], a[3]}, B = {b[0], b[1], b[2], b[3]};
    const camp X = {x[0], x[1], x[2], x[3]}, Y = {y[0], y[1], y[2], y[3]};
    const camp o = rmad2(A, X, B, Y);
    out[0] = o.rh; out[1] = o.rl; out[2] = o.ih; out[3] = o.il;
}
void shim_cmul(const float *d, const float *x, float *out) {
    const ccst D = {d[0], d[1], d[2], d[3]};
    const camp X = {x[0], x[1], x[2], x[3]};
    const camp o = cmul(D, X);
    out[0] = o.rh; out[1] = o.rl; out[2] = o.ih; out[3] = o.il;
}
void shim_butterfly(float *x, float *y) {
    camp X = {x[0], x[1], x[2], x[3]}, Y = {y[0], y[1], y[2], y[3]};
    butterfly(X, Y);
    x[0] = X.rh; x[1] = X.rl; x[2] = X.ih; x[3] = X.il;
    y[0] = Y.rh; y[1] = Y.rl; y[2] = Y.ih; y[3] = Y.il;
}
void shim_mul1(float xh, float xl, float ch, float cl, float *h, float *l) { mul1(xh, xl, ch, cl, *h, *l); }
void shim_split_const(double c, float *h, float *l) { split_const(c, *h, *l); }
}
