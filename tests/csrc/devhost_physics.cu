// Pointwise physics evaluated in a device kernel and on the host from the same
// source: values and dual tangents must agree to rounding.  Guards against
// device-only miscompilation of the dual arithmetic (a run-time index into a
// local array of dual numbers once gave a wrong tangent on the device only).
// Exit status 0 iff every max |host - device| <= 1e-13.
#include <cmath>
#include <cstdio>
#include <cstdlib>

#include "dg_common.cuh"
using namespace dgk;
typedef Dual<double> DD;

template <int D>
struct In {
  double u[D + 2], du[D + 2], g[D + 2][D], dg[D + 2][D], uR[D + 2], duR[D + 2];
};
template <int D>
struct Out {
  double Ft[D + 2][D], dFt[D + 2][D], fp[D][D + 2], dfp[D][D + 2], Dh[D][D + 2][D], dDh[D][D + 2][D],
      Gn[D][D + 2], dGn[D][D + 2];
};

template <int D>
__host__ __device__ void compute(const In<D>& in, Out<D>& o, const Phys<double>& ph) {
  constexpr int M = D + 2;
  DD u[M], g[M][D], F[M][D], uR[M], gR[M][D];
  for (int v = 0; v < M; ++v) {
    u[v] = DD(in.u[v], in.du[v]);
    uR[v] = DD(in.uR[v], in.duR[v]);
    for (int k = 0; k < D; ++k) {
      g[v][k] = DD(in.g[v][k], in.dg[v][k]);
      gR[v][k] = DD(0.5 * in.g[v][k], -in.dg[v][k]);
    }
  }
  flux_total<D, DD, double>(u, g, F, ph);
  for (int v = 0; v < M; ++v)
    for (int k = 0; k < D; ++k) {
      o.Ft[v][k] = F[v][k].v;
      o.dFt[v][k] = F[v][k].d;
    }
  for (int k = 0; k < D; ++k) {
    DD fp[M], GLn[M], GRn[M], DL[M][D], DR[M][D];
    face_point_k<D, DD, double>(k, u, g, uR, gR, ph, fp, GLn, GRn, DL, DR);
    for (int v = 0; v < M; ++v) {
      o.fp[k][v] = fp[v].v;
      o.dfp[k][v] = fp[v].d;
      o.Gn[k][v] = GLn[v].v - GRn[v].v;
      o.dGn[k][v] = GLn[v].d + 2.0 * GRn[v].d;
      for (int kk = 0; kk < D; ++kk) {
        o.Dh[k][v][kk] = DL[v][kk].v + DR[v][kk].v;
        o.dDh[k][v][kk] = DL[v][kk].d - DR[v][kk].d;
      }
    }
  }
}

template <int D>
__global__ void kern(In<D> in, Out<D>* o, Phys<double> ph) {
  compute<D>(in, *o, ph);
}

template <int D>
int run() {
  Phys<double> ph;
  ph.gamma = 1.4; ph.gm1 = 0.4; ph.Pr = 0.72; ph.mu = 0.05; ph.Rgas = 1; ph.eta = 7; ph.roe_delta = 0.1;
  ph.kappa = ph.mu * 1.4 / (0.4 * 0.72);
  In<D> in;
  srand(3);
  auto r = [] { return rand() / (double)RAND_MAX - 0.5; };
  for (int v = 0; v < D + 2; ++v) {
    in.u[v] = (v == 0) ? 1.1 : (v == D + 1 ? 2.8 : 0.3 * r());
    in.uR[v] = in.u[v] * (1 + 0.05 * r());
    in.du[v] = r();
    in.duR[v] = r();
    for (int k = 0; k < D; ++k) {
      in.g[v][k] = r();
      in.dg[v][k] = r();
    }
  }
  in.u[1] = 0.01;          // small normal speed: the entropy-fix branch of the Roe flux
  Out<D> h, d, *dptr;
  compute<D>(in, h, ph);
  if (cudaMalloc(&dptr, sizeof(Out<D>)) != cudaSuccess) return 2;
  kern<D><<<1, 1>>>(in, dptr, ph);
  if (cudaMemcpy(&d, dptr, sizeof(Out<D>), cudaMemcpyDeviceToHost) != cudaSuccess) return 2;
  cudaFree(dptr);
  const double* a = (const double*)&h;
  const double* b = (const double*)&d;
  size_t n = sizeof(Out<D>) / sizeof(double);
  double e = 0;
  for (size_t i = 0; i < n; ++i) e = fmax(e, fabs(a[i] - b[i]) / fmax(1.0, fabs(a[i])));
  printf("D=%d max |host - device| = %.3e over %zu values\n", D, e, n);
  return e <= 1e-13 ? 0 : 1;
}

int main() { return run<2>() | run<3>(); }
