// Host harness of the CUDA path's raster functions (vlb_raster.cuh compiled
// for the CPU).  Reads lines "X Y R i j" and prints, for FP32 and FP64, the
// cell class and solid fraction of cell (i, j) against disk (X, Y, R), with
// the particle record set up as the lattice kernel does for a tile at (0, 0).
#include <cmath>
#include <cstdio>

#include "vlb_raster.cuh"

template <class C>
static vlb::PartTile<C> make(double X, double Y, double R) {
  vlb::PartTile<C> q{};
  const long long Q = 1ll << vlb::QBITS;
  q.xq = std::llrint(X * double(Q));
  q.yq = std::llrint(Y * double(Q));
  const long long rq = std::llrint(R * double(Q));
  q.rq2 = rq * rq;
  q.xh = C(X); q.xl = C(X - double(q.xh));
  q.yh = C(Y); q.yl = C(Y - double(q.yh));
  q.r = C(R);
  q.far2 = C((R + 0.75) * (R + 0.75));
  q.near2 = R > 0.75 ? C((R - 0.75) * (R - 0.75)) : C(-1);
  return q;
}

int main() {
  double X, Y, R;
  int i, j;
  while (std::scanf("%lf %lf %lf %d %d", &X, &Y, &R, &i, &j) == 5) {
    float f32;
    double f64;
    const int c32 = vlb::cell_fraction(i, j, make<float>(X, Y, R), f32);
    const int c64 = vlb::cell_fraction(i, j, make<double>(X, Y, R), f64);
    std::printf("%d %.9e %d %.17e\n", c32, (double)f32, c64, f64);
  }
  return 0;
}
