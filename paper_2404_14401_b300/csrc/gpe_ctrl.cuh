// gpe_ctrl.cuh -- the arguments of one pass evaluated on the device (sm_103a),
// for the kernels that run many passes per launch: the persistent batch
// (gpe_batch.cu) and the cooperative single-grid kernel (gpe_coop.cu).  D is
// any descriptor with the context's potential parameters and control points
// (BatchCtx, CoopArgs).
#pragma once

#include <cuda_runtime.h>

#include "../../include/gpe.h"
#include "gpe_internal.h"

namespace gpe {

// ------------------------------------------------------------------ per-pass arguments
// The piecewise-linear control v(t), the phase and the reduction arguments of
// a pass at time t, computed as the host scheduler computes them (the same
// double operations, without contraction into fused multiply-adds).
template <class D> __device__ double ctrl_value(const D &c, double t)
{
    const int n = c.nctrl;
    if (n == 0) return 1.0;
    if (t <= c.ctrl_t[0]) return c.ctrl_v[0];
    if (t >= c.ctrl_t[n - 1]) return c.ctrl_v[n - 1];
    int lo = 0, hi = n - 1;                        // ctrl_t[lo] < t < ctrl_t[hi]
    while (hi - lo > 1) {
        const int mid = (lo + hi) / 2;
        if (c.ctrl_t[mid] < t) lo = mid; else hi = mid;
    }
    const double f = __ddiv_rn(__dsub_rn(t, c.ctrl_t[lo]), __dsub_rn(c.ctrl_t[hi], c.ctrl_t[lo]));
    return __dadd_rn(c.ctrl_v[lo], __dmul_rn(f, __dsub_rn(c.ctrl_v[hi], c.ctrl_v[lo])));
}

template <class D> __device__ double eta_dev(const D &c, double t)
{
    return c.ctrl_target == GPE_CTRL_ETA ? ctrl_value(c, t) : c.eta;
}

template <class D> __device__ PhaseArgs phase_dev(const D &c, double t, double h)
{
    const double ls = c.ctrl_target == GPE_CTRL_LATTICE ? ctrl_value(c, t) : 1.0;
    const double eta = eta_dev(c, t);
    PhaseArgs a;
    a.h = (float)h;
    a.a_latx = (float)__dmul_rn(c.lat_V0x, ls);
    a.a_laty = (float)__dmul_rn(c.lat_V0y, ls);
    a.a_pump = (c.cavity && c.pump_lattice && c.U0 != 0.0) ? (float)__ddiv_rn(__dmul_rn(eta, eta), c.U0) : 0.f;
    a.U0 = c.cavity ? (float)c.U0 : 0.f;
    a.two_eta = c.cavity ? (float)__dmul_rn(2.0, eta) : 0.f;
    a.use_alpha = c.cavity ? 1 : 0;
    return a;
}

template <class D> __device__ RedArgs red_dev(const D &c, double t)
{
    RedArgs r;
    r.eta = eta_dev(c, t);
    r.U0 = c.U0;
    r.dc = c.dc;
    r.kappa = c.kappa;
    r.N = c.N;
    r.dxdy = c.dxdy;
    r.cavity = c.cavity;
    r.probe_omega = c.probe_omega;
    r.probe_delta = c.probe_delta;
    r.probe_phi = c.probe_phi;
    r.t = t;
    return r;
}

}  // namespace gpe
