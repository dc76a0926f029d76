// Simplex quadrature rules of the discrete problem (barycentric points, weights
// summing to one):
//  tetrahedron degree 2 (4 points): (alpha, beta, beta, beta) and permutations,
//      alpha = (5 + 3 sqrt 5)/20, beta = (5 - sqrt 5)/20, weights 1/4;
//  tetrahedron degree 5 (14 points): the fully symmetric rule of Walkington
//      (orbits (a,a,a,1-3a) for two a, and (c,c,1/2-c,1/2-c));
//  triangle degree 2 (3 points): (2/3, 1/6, 1/6) and permutations, weights 1/3;
//  triangle degree 5 (7 points, Radon): centroid 9/40 and two orbits
//      a = (6 -+ sqrt 15)/21 with weights (155 -+ sqrt 15)/1200.
// The orbit order (lexicographic over distinct permutations) is fixed so that
// point k means the same point everywhere in the library.
#include <algorithm>
#include <array>
#include <cmath>
#include <vector>

#include "fill.h"

namespace vie {

template <int D>
static void orbit(std::array<double, D> v, std::vector<std::array<double, D>> &out) {
    std::sort(v.begin(), v.end());
    do {
        out.push_back(v);
    } while (std::next_permutation(v.begin(), v.end()));
}

void tet_rule2(double (*pts)[4], double *w) {
    const double s5 = std::sqrt(5.0);
    const double al = (5.0 + 3.0 * s5) / 20.0, be = (5.0 - s5) / 20.0;
    std::vector<std::array<double, 4>> o;
    orbit<4>({al, be, be, be}, o);
    for (int k = 0; k < 4; ++k) {
        if (pts) for (int j = 0; j < 4; ++j) pts[k][j] = o[k][j];
        if (w) w[k] = 0.25;
    }
}

void tet_rule5(double (*pts)[4], double *w) {
    const double a1 = 0.0927352503108912264, w1 = 0.0734930431163619495;
    const double a2 = 0.3108859192633006097, w2 = 0.1126879257180158507;
    const double c3 = 0.0455037041256496494, w3 = 0.0425460207770814664;
    std::vector<std::array<double, 4>> o;
    std::vector<double> ww;
    orbit<4>({a1, a1, a1, 1.0 - 3.0 * a1}, o);
    ww.resize(o.size(), w1);
    orbit<4>({a2, a2, a2, 1.0 - 3.0 * a2}, o);
    ww.resize(o.size(), w2);
    orbit<4>({c3, c3, 0.5 - c3, 0.5 - c3}, o);
    ww.resize(o.size(), w3);
    for (int k = 0; k < 14; ++k) {
        if (pts) for (int j = 0; j < 4; ++j) pts[k][j] = o[k][j];
        if (w) w[k] = ww[k];
    }
}

void tri_rule2(double (*pts)[3], double *w) {
    std::vector<std::array<double, 3>> o;
    orbit<3>({2.0 / 3.0, 1.0 / 6.0, 1.0 / 6.0}, o);
    for (int k = 0; k < 3; ++k) {
        if (pts) for (int j = 0; j < 3; ++j) pts[k][j] = o[k][j];
        if (w) w[k] = 1.0 / 3.0;
    }
}

void tri_rule5(double (*pts)[3], double *w) {
    const double s15 = std::sqrt(15.0);
    const double a1 = (6.0 - s15) / 21.0, a2 = (6.0 + s15) / 21.0;
    const double w1 = (155.0 - s15) / 1200.0, w2 = (155.0 + s15) / 1200.0;
    std::vector<std::array<double, 3>> o;
    std::vector<double> ww;
    o.push_back({1.0 / 3.0, 1.0 / 3.0, 1.0 / 3.0});
    ww.push_back(9.0 / 40.0);
    orbit<3>({a1, a1, 1.0 - 2.0 * a1}, o);
    ww.resize(o.size(), w1);
    orbit<3>({a2, a2, 1.0 - 2.0 * a2}, o);
    ww.resize(o.size(), w2);
    for (int k = 0; k < 7; ++k) {
        if (pts) for (int j = 0; j < 3; ++j) pts[k][j] = o[k][j];
        if (w) w[k] = ww[k];
    }
}

}  // namespace vie
