// Host set-up of the Ewald tables of one incidence (ewald_tables.cpp).
#pragma once
#include <vector>

#include "ewald_params.h"

namespace vie {

// Ewald parameters and tables of one incidence; status as vie_status;
// split_mult > 0: the FP32 tables' Ewald split multiplier (else the default)
int build_ewald_tables(double a, double b, double k0, double kx, double ky, double z_extent, bool fp64,
                       EwaldTables &E, std::vector<double> *orders, const char **why,
                       double split_mult = 0.0);

}  // namespace vie
