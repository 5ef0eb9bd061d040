// Host numerics of the setup stage (see setup_host.cpp).
#pragma once

#include <vector>

namespace klecgc {

void kl_modes_1d(double corr_len, double sigma, int count, std::vector<double>& lam,
                 std::vector<double>& omega, std::vector<int>& parity);
// Top-`count` 2D separable modes: eigenvalues lam, 1D mode indices (mi, mj)
// into the unit-variance 1D pairs (mu, omega, parity).
void kl_modes_2d(double corr_len, double sigma, int count, std::vector<double>& lam,
                 std::vector<int>& mi, std::vector<int>& mj, std::vector<double>& mu,
                 std::vector<double>& omega, std::vector<int>& parity);
double kl_phi_1d(double x, double w, int parity);
std::vector<int> gpc_multi_indices(int M, int p);

}  // namespace klecgc
