// mp_gravity.cu -- gravitational source terms of the fluid balance equations
// (GenASiS II, Sec. 3, Eq. (BalancedVariablesGravitational)) from a potential
// on the solver's mesh:
//
//   grad[a] = d(Phi)/dx^a   (x = r, theta, phi; coordinate derivatives)
//   S[a]    = -rho grad[a]  (momentum source, covariant components)
//   E       = -rho v^a grad[a]  (energy source; v contravariant)
//
// Each derivative is the simplest centred difference, over the two nearest
// cells along the coordinate (the rule the paper states with the sources):
// (Phi[hi] - Phi[lo]) / (x_c[hi] - x_c[lo]) with cell centres at coordinate
// midpoints.  phi wraps around when the azimuthal edges span 2 pi; at the ends
// of r, theta (and of a shorter azimuthal range) the two nearest cells are the
// cell itself and its one neighbour.  A single cell along a coordinate, or two
// azimuthal cells on a full circle, give a zero derivative.
//
// One block per (shell, polar cell) row, threads along phi (rows of fewer than 32 cells:
// one thread per cell over the flattened mesh).  The potential is
// read through the cache (each value serves the six neighbouring differences:
// rows j +- 1 and shells i +- 1 are read by nearby blocks while they are still
// in L2); density, velocity and the outputs stream once (evict-first).  All
// arithmetic is float64.
#include <cmath>

#include "mp_internal.h"
#include "ptx.cuh"

namespace mp {

namespace {

__global__ void __launch_bounds__(256) k_gravity(const double *__restrict__ phi, const double *__restrict__ rho,
                                                 const double *__restrict__ v, double *__restrict__ grad,
                                                 double *__restrict__ S, double *__restrict__ E,
                                                 const GradStencil *__restrict__ st, int n_r, int n_t, int n_p,
                                                 long long N)
{
    const long long row = blockIdx.x;  // i n_t + j
    const int i = (int)(row / n_t), j = (int)(row - (long long)i * n_t);
    const GradStencil gr = st[i], gt = st[n_r + j];
    const GradStencil *sp = st + n_r + n_t;
    const double *p_row = phi + row * n_p;
    const double *p_rlo = phi + ((long long)gr.lo * n_t + j) * n_p, *p_rhi = phi + ((long long)gr.hi * n_t + j) * n_p;
    const double *p_tlo = phi + ((long long)i * n_t + gt.lo) * n_p, *p_thi = phi + ((long long)i * n_t + gt.hi) * n_p;
    for (int k = threadIdx.x; k < n_p; k += blockDim.x) {
        const GradStencil gp = sp[k];
        const long long c = row * n_p + k;
        const double g0 = (__ldg(p_rhi + k) - __ldg(p_rlo + k)) * gr.w;
        const double g1 = (__ldg(p_thi + k) - __ldg(p_tlo + k)) * gt.w;
        const double g2 = (__ldg(p_row + gp.hi) - __ldg(p_row + gp.lo)) * gp.w;
        if (grad) {
            __stcs(grad + c, g0);
            __stcs(grad + N + c, g1);
            __stcs(grad + 2 * N + c, g2);
        }
        const double nr = -__ldcs(rho + c);
        if (S) {
            const double s0 = nr * g0, s1 = nr * g1, s2 = nr * g2;
            __stcs(S + c, s0);
            __stcs(S + N + c, s1);
            __stcs(S + 2 * N + c, s2);
            // E = v^a S_a: the products are already there (12 float64 operations a cell, not 13)
            if (E) __stcs(E + c, fma(__ldcs(v + 2 * N + c), s2, fma(__ldcs(v + N + c), s1, __ldcs(v + c) * s0)));
        } else if (E) {
            const double vg = fma(__ldcs(v + 2 * N + c), g2, fma(__ldcs(v + N + c), g1, __ldcs(v + c) * g0));
            __stcs(E + c, nr * vg);
        }
    }
}

// The same sources with one thread per cell over the flattened mesh, for rows shorter than
// a warp (2-D meshes have one azimuthal cell: a block per row would hold one busy thread).
__global__ void __launch_bounds__(256) k_gravity_flat(const double *__restrict__ phi, const double *__restrict__ rho,
                                                      const double *__restrict__ v, double *__restrict__ grad,
                                                      double *__restrict__ S, double *__restrict__ E,
                                                      const GradStencil *__restrict__ st, int n_r, int n_t,
                                                      int n_p, long long N)
{
    const long long c = (long long)blockIdx.x * blockDim.x + threadIdx.x;
    if (c >= N) return;
    const long long row = c / n_p;
    const int k = (int)(c - row * n_p);
    const int i = (int)(row / n_t), j = (int)(row - (long long)i * n_t);
    const GradStencil gr = st[i], gt = st[n_r + j], gp = st[n_r + n_t + k];
    const double *p_r = phi + (long long)j * n_p + k, *p_t = phi + (long long)i * n_t * n_p + k;
    const double g0 = (__ldg(p_r + (long long)gr.hi * n_t * n_p) - __ldg(p_r + (long long)gr.lo * n_t * n_p)) * gr.w;
    const double g1 = (__ldg(p_t + (long long)gt.hi * n_p) - __ldg(p_t + (long long)gt.lo * n_p)) * gt.w;
    const double g2 = (__ldg(phi + row * n_p + gp.hi) - __ldg(phi + row * n_p + gp.lo)) * gp.w;
    if (grad) {
        grad[c] = g0;
        grad[N + c] = g1;
        grad[2 * N + c] = g2;
    }
    const double nr = -rho[c];
    if (S) {
        const double s0 = nr * g0, s1 = nr * g1, s2 = nr * g2;
        S[c] = s0;
        S[N + c] = s1;
        S[2 * N + c] = s2;
        if (E) E[c] = fma(v[2 * N + c], s2, fma(v[N + c], s1, v[c] * s0));
    } else if (E) {
        E[c] = nr * fma(v[2 * N + c], g2, fma(v[N + c], g1, v[c] * g0));
    }
}

// lo, hi, 1/dx per cell along one axis (the rule of the file header)
void axis_stencil(const std::vector<double> &e, bool periodic, GradStencil *out)
{
    const int n = (int)e.size() - 1;
    std::vector<double> xc(n);
    for (int i = 0; i < n; ++i) xc[i] = 0.5 * (e[i] + e[i + 1]);
    const double period = e[n] - e[0];
    for (int i = 0; i < n; ++i) {
        int lo, hi;
        double dx;
        if (n == 1) {
            lo = hi = 0;
            dx = 0.0;
        } else if (periodic) {
            lo = (i + n - 1) % n;
            hi = (i + 1) % n;
            const double x_lo = xc[lo] - (i == 0 ? period : 0.0);
            const double x_hi = xc[hi] + (i == n - 1 ? period : 0.0);
            dx = (lo == hi) ? 0.0 : x_hi - x_lo;
        } else {
            lo = i > 0 ? i - 1 : 0;
            hi = i < n - 1 ? i + 1 : n - 1;
            dx = xc[hi] - xc[lo];
        }
        out[i].lo = lo;
        out[i].hi = hi;
        out[i].w = dx != 0.0 ? 1.0 / dx : 0.0;
    }
}

}  // namespace

cudaError_t gravity_prepare(mp_mesh *m)
{
    constexpr double kTwoPi = 6.283185307179586477;
    std::vector<GradStencil> h((size_t)m->n_r + m->n_t + m->n_p);
    axis_stencil(m->h_r, false, h.data());
    axis_stencil(m->h_th, false, h.data() + m->n_r);
    const double span = m->h_ph.back() - m->h_ph.front();
    const bool full_circle = std::fabs(span - kTwoPi) <= 1e-12 * kTwoPi;
    axis_stencil(m->h_ph, full_circle, h.data() + m->n_r + m->n_t);
    cudaError_t e = cudaMalloc(reinterpret_cast<void **>(&m->d_gst), h.size() * sizeof(GradStencil));
    if (e != cudaSuccess) return e;
    m->device_bytes += h.size() * sizeof(GradStencil);
    return cudaMemcpy(m->d_gst, h.data(), h.size() * sizeof(GradStencil), cudaMemcpyHostToDevice);
}

cudaError_t launch_gravity(mp_mesh *m, const double *phi, const double *rho, const double *v, double *grad, double *S,
                           double *E)
{
    cudaEvent_t ev;
    prof_begin(m, "gravity_sources", &ev);
    if (m->n_p < 32) {
        k_gravity_flat<<<(unsigned)((m->N + 255) / 256), 256, 0, m->stream>>>(phi, rho, v, grad, S, E, m->d_gst, m->n_r,
                                                                              m->n_t, m->n_p, m->N);
    } else {
        const int threads = std::min(256, 32 * ((m->n_p + 31) / 32));
        k_gravity<<<(unsigned)m->R, threads, 0, m->stream>>>(phi, rho, v, grad, S, E, m->d_gst, m->n_r, m->n_t,
                                                             m->n_p, m->N);
    }
    prof_end(m, "gravity_sources", ev);
    return cudaGetLastError();
}

}  // namespace mp
