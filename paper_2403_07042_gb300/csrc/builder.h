// Host-side model builder: basis enumeration, dense projected H, monomial jump tables.
#pragma once

#include <complex>
#include <cstdint>
#include <string>
#include <unordered_map>
#include <vector>

#include "qed.h"

namespace qed {

using cplx = std::complex<double>;

struct Layout {
    std::vector<int> radix;          // per digit
    std::vector<char> counted;       // digit counts towards the excitation number
    std::vector<int> photon_digit;   // per cavity
    std::vector<int> atom_digit;     // per atom
    std::vector<int> atom_cavity;    // per atom
    std::vector<int> extra_digit;    // per extra two-level DOF
    int n_digits() const { return (int)radix.size(); }
};

// One jump operator entry: A_j |src> = coef |dst> (monomial: one entry per column).
struct JumpEntry {
    int32_t jump;
    int64_t src;
    int64_t dst;
    double coef;
};

struct HostModel {
    // specification copy
    int32_t n_cavities = 0, n_extra = 0, basis_kind = 0, excitation_cap = 0;
    int64_t dim_cap = 0;
    double omega_c = 1.0, omega_a = 1.0;
    std::vector<int32_t> atoms_per_cavity, n_max;
    std::vector<double> g, zeta, extra_tunnel, gamma;
    std::vector<int32_t> bond_i, bond_j, jump_kind, jump_site;

    Layout layout;
    int64_t dim = 0;
    std::vector<uint8_t> digits;                 // dim x n_digits
    std::unordered_map<std::string, int64_t> index;

    // H_kl = coefficient * unit of each nonzero; `param` tells which spec entry
    // multiplies it (0 diagonal, 1 g, 2 zeta, 3 extra_tunnel) and `which` its index.
    struct HEntry { int64_t row, col; double unit; int8_t param; int32_t which; };
    std::vector<HEntry> h_entries;

    std::vector<JumpEntry> jumps;               // all jumps, all entries
    std::vector<double> anti_diag;              // d_k = sum_j gamma_j (A_j^+ A_j)_kk
};

// Validates and copies a spec; builds basis, H entries and jump entries.
// Returns QED_OK or an error code with `err` describing it.
qed_status build_host_model(const qed_spec *spec, HostModel &hm, std::string &err,
                            bool operators = true);

std::string state_key(const uint8_t *digits, int n_digits);

// The model on the basis states `keep` (increasing indices of src's basis): H and every
// A_j projected onto them (P H P, P A_j P), renumbered; d_k recomputed from the kept jump
// entries.  Returns false with `err` set for an empty or unsorted list.
bool restrict_host_model(const HostModel &src, const std::vector<int64_t> &keep, HostModel &dst,
                         std::string &err);

// Dense row-major complex H.
void dense_hamiltonian(const HostModel &hm, std::vector<cplx> &H);

// Value of the parameter multiplying an H entry.
double entry_coefficient(const HostModel &hm, const HostModel::HEntry &e);

constexpr int64_t kMaxDim = 32768;

}  // namespace qed
