// Host-side table generators (double precision); see host_tables.cpp.
#pragma once
#include <vector>

#include "common.cuh"

namespace purify {
double kb_ft(double nu, int J, int K, double beta);
std::vector<double> correction_axis(int n, int K, int J, double beta);
KbPoly fit_kb_poly(int J, double beta, int deg);
int kb_poly_degree(int J);
std::vector<double> twiddles(int K);
std::vector<double> daubechies(int p);
}  // namespace purify
