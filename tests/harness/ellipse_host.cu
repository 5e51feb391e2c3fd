// Host harness of the CUDA path's ellipse raster functions (vlb_raster.cuh
// compiled for the CPU).  Reads lines "X Y a b c s i j" (centre, semi-axes,
// cosine and sine of the major axis's angle, cell) and prints the class and
// the FP64 area of the ellipse in cell [i, i+1] x [j, j+1] as the FP64
// lattice kernel and the band pass compute them.
#include <cstdio>

#include "vlb_raster.cuh"

int main() {
  double X, Y, a, b, c, s;
  int i, j;
  while (std::scanf("%lf %lf %lf %lf %lf %lf %d %d", &X, &Y, &a, &b, &c, &s, &i, &j) == 8) {
    const int cls = vlb::ellipse_cell_class(i, j, X, Y, a, b, c, s);
    const double ar = vlb::ellipse_cell_area(i, j, X, Y, a, b, c, s);
    std::printf("%d %.17e\n", cls, ar);
  }
  return 0;
}
