// Host-side model builder (Sec. 2, first point): digit-string basis states, the dense
// projected Hamiltonian of Eqs. (8b)-(8d) and (12), and the jump operators of Eq. (3)
// as monomial tables (every operator here maps a basis state to at most one state).
#include "builder.h"

#include <algorithm>
#include <cmath>
#include <functional>

namespace qed {

std::string state_key(const uint8_t *d, int n) {
    // sparse key: (position, value) of the nonzero digits, so long one-excitation
    // states hash cheaply
    std::string key;
    for (int i = 0; i < n; ++i) {
        if (d[i]) {
            key.push_back((char)(i & 0xff));
            key.push_back((char)((i >> 8) & 0xff));
            key.push_back((char)((i >> 16) & 0xff));
            key.push_back((char)d[i]);
        }
    }
    return key;
}

namespace {

bool fail(std::string &err, const std::string &msg) {
    err = msg;
    return false;
}

bool copy_spec(const qed_spec *s, HostModel &hm, std::string &err) {
    if (!s) return fail(err, "spec is NULL");
    if (s->n_cavities < 0 || s->n_extra < 0 || s->n_bonds < 0 || s->n_jumps < 0)
        return fail(err, "negative count in spec");
    if (s->n_cavities > 0 && (!s->atoms_per_cavity || !s->n_max))
        return fail(err, "atoms_per_cavity / n_max missing");
    hm.n_cavities = s->n_cavities;
    hm.n_extra = s->n_extra;
    hm.basis_kind = s->basis_kind;
    hm.excitation_cap = s->excitation_cap;
    hm.dim_cap = s->dim_cap;
    hm.omega_c = s->omega_c;
    hm.omega_a = s->omega_a;
    if (!std::isfinite(hm.omega_c) || !std::isfinite(hm.omega_a)) return fail(err, "non-finite omega");
    int n_atoms = 0;
    for (int c = 0; c < s->n_cavities; ++c) {
        if (s->atoms_per_cavity[c] < 0 || s->atoms_per_cavity[c] > 64) return fail(err, "atoms_per_cavity out of range");
        if (s->n_max[c] < 0 || s->n_max[c] > 200) return fail(err, "n_max out of range");
        hm.atoms_per_cavity.push_back(s->atoms_per_cavity[c]);
        hm.n_max.push_back(s->n_max[c]);
        n_atoms += s->atoms_per_cavity[c];
    }
    if (n_atoms > 0 && !s->g) return fail(err, "g missing");
    hm.g.assign(s->g, s->g + n_atoms);
    for (double v : hm.g) if (!std::isfinite(v)) return fail(err, "non-finite g");
    if (s->n_bonds > 0 && (!s->bond_ij || !s->zeta)) return fail(err, "bonds missing");
    for (int b = 0; b < s->n_bonds; ++b) {
        int i = s->bond_ij[2 * b], j = s->bond_ij[2 * b + 1];
        if (i < 0 || j < 0 || i >= s->n_cavities || j >= s->n_cavities || i == j)
            return fail(err, "bond cavity index out of range");
        if (!std::isfinite(s->zeta[b])) return fail(err, "non-finite zeta");
        hm.bond_i.push_back(i);
        hm.bond_j.push_back(j);
        hm.zeta.push_back(s->zeta[b]);
    }
    if (s->n_extra > 0) {
        if (!s->extra_tunnel) return fail(err, "extra_tunnel missing");
        hm.extra_tunnel.assign(s->extra_tunnel, s->extra_tunnel + s->n_extra);
    }
    if (s->n_jumps > 0 && (!s->jump_kind || !s->jump_site || !s->gamma)) return fail(err, "jumps missing");
    for (int j = 0; j < s->n_jumps; ++j) {
        int k = s->jump_kind[j], site = s->jump_site[j];
        double gm = s->gamma[j];
        if (!(gm >= 0.0) || !std::isfinite(gm)) return fail(err, "jump rate must be finite and >= 0");
        int lim = k == QED_JUMP_A || k == QED_JUMP_LEAK ? s->n_cavities
                : k == QED_JUMP_SIGMA ? n_atoms : k == QED_JUMP_DEPHASE ? s->n_extra : -1;
        if (lim < 0) return fail(err, "unknown jump kind");
        if (site < 0 || site >= lim) return fail(err, "jump site out of range");
        hm.jump_kind.push_back(k);
        hm.jump_site.push_back(site);
        hm.gamma.push_back(gm);
    }
    return true;
}

void make_layout(HostModel &hm) {
    Layout &L = hm.layout;
    for (int c = 0; c < hm.n_cavities; ++c) {
        L.photon_digit.push_back((int)L.radix.size());
        L.radix.push_back(hm.n_max[c] + 1);
        L.counted.push_back(1);
        for (int a = 0; a < hm.atoms_per_cavity[c]; ++a) {
            L.atom_digit.push_back((int)L.radix.size());
            L.atom_cavity.push_back(c);
            L.radix.push_back(2);
            L.counted.push_back(1);
        }
    }
    for (int x = 0; x < hm.n_extra; ++x) {
        L.extra_digit.push_back((int)L.radix.size());
        L.radix.push_back(2);
        L.counted.push_back(0);
    }
}

// Emits, in mixed-radix order, every digit string whose excitation count lies in
// [lo, hi]; stops (returns false) once `limit` states have been produced.
bool enumerate_range(const Layout &L, int lo, int hi, int64_t limit, std::vector<uint8_t> &out,
                     int64_t &count) {
    const int n = L.n_digits();
    std::vector<int> suffix(n + 1, 0);
    for (int i = n - 1; i >= 0; --i) suffix[i] = suffix[i + 1] + (L.counted[i] ? L.radix[i] - 1 : 0);
    std::vector<uint8_t> cur(n, 0);
    bool ok = true;
    // explicit stack of (digit, value, used) so deep digit strings need no recursion
    std::vector<int> val(n + 1, -1), used(n + 1, 0);
    int i = 0;
    used[0] = 0;
    val[0] = -1;
    while (i >= 0) {
        if (i == n) {
            if (used[n] >= lo && used[n] <= hi) {
                if (count >= limit) { ok = false; break; }
                out.insert(out.end(), cur.begin(), cur.end());
                ++count;
            }
            --i;
            continue;
        }
        int v = ++val[i];
        if (v >= L.radix[i]) {
            cur[i] = 0;
            val[i] = -1;
            --i;
            continue;
        }
        int u = used[i] + (L.counted[i] ? v : 0);
        if (u > hi) {  // larger values only add excitations
            cur[i] = 0;
            val[i] = -1;
            --i;
            continue;
        }
        if (u + suffix[i + 1] < lo) continue;
        cur[i] = (uint8_t)v;
        used[i + 1] = u;
        val[i + 1] = -1;
        ++i;
    }
    return ok;
}

bool enumerate_basis(HostModel &hm, std::string &err) {
    const Layout &L = hm.layout;
    const int n = L.n_digits();
    hm.digits.clear();
    int64_t count = 0;
    int max_exc = 0;
    for (int i = 0; i < n; ++i) if (L.counted[i]) max_exc += L.radix[i] - 1;
    switch (hm.basis_kind) {
    case QED_BASIS_FULL:
        if (!enumerate_range(L, 0, max_exc, kMaxDim, hm.digits, count))
            return fail(err, "basis larger than the supported maximum dimension");
        break;
    case QED_BASIS_CAP:
        if (hm.excitation_cap < 0) return fail(err, "negative excitation_cap");
        if (!enumerate_range(L, 0, hm.excitation_cap, kMaxDim, hm.digits, count))
            return fail(err, "basis larger than the supported maximum dimension");
        break;
    case QED_BASIS_SECTOR:
        if (hm.excitation_cap < 0) return fail(err, "negative excitation_cap");
        if (!enumerate_range(L, hm.excitation_cap, hm.excitation_cap, kMaxDim, hm.digits, count))
            return fail(err, "basis larger than the supported maximum dimension");
        break;
    case QED_BASIS_FIRST_D: {
        if (hm.dim_cap < 1 || hm.dim_cap > kMaxDim) return fail(err, "dim_cap out of range");
        for (int e = 0; e <= max_exc && count < hm.dim_cap; ++e) {
            std::vector<uint8_t> sec;
            int64_t c2 = 0;
            enumerate_range(L, e, e, hm.dim_cap - count, sec, c2);
            hm.digits.insert(hm.digits.end(), sec.begin(), sec.end());
            count += c2;
        }
        if (count < hm.dim_cap) return fail(err, "dim_cap exceeds the product space");
        break;
    }
    case QED_BASIS_SINGLE_G: {
        if (hm.n_extra) return fail(err, "the ground + single-excitation basis takes no extra digits");
        std::vector<uint8_t> row(n, 0);
        hm.digits.insert(hm.digits.end(), row.begin(), row.end());
        count = 1;
        int atom = 0;
        for (int c = 0; c < hm.n_cavities; ++c) {
            if (hm.n_max[c] >= 1) {
                std::fill(row.begin(), row.end(), 0);
                row[L.photon_digit[c]] = 1;
                hm.digits.insert(hm.digits.end(), row.begin(), row.end());
                ++count;
            }
            for (int a = 0; a < hm.atoms_per_cavity[c]; ++a, ++atom) {
                std::fill(row.begin(), row.end(), 0);
                row[L.atom_digit[atom]] = 1;
                hm.digits.insert(hm.digits.end(), row.begin(), row.end());
                ++count;
            }
            if (count > kMaxDim) return fail(err, "basis larger than the supported maximum dimension");
        }
        break;
    }
    default:
        return fail(err, "unknown basis kind");
    }
    if (count == 0) return fail(err, "empty basis");
    hm.dim = count;
    hm.index.clear();
    hm.index.reserve((size_t)count * 2);
    for (int64_t k = 0; k < count; ++k) hm.index.emplace(state_key(&hm.digits[(size_t)k * n], n), k);
    return true;
}

int64_t find(const HostModel &hm, const std::vector<uint8_t> &d) {
    auto it = hm.index.find(state_key(d.data(), (int)d.size()));
    return it == hm.index.end() ? -1 : it->second;
}

void build_hamiltonian(HostModel &hm) {
    const Layout &L = hm.layout;
    const int n = L.n_digits();
    hm.h_entries.clear();
    std::vector<uint8_t> t(n);
    auto emit = [&](int64_t col, double unit, int8_t param, int32_t which) {
        int64_t row = find(hm, t);
        if (row >= 0) hm.h_entries.push_back({row, col, unit, param, which});
    };
    for (int64_t k = 0; k < hm.dim; ++k) {
        const uint8_t *d = &hm.digits[(size_t)k * n];
        double e = 0.0;
        for (int c = 0; c < hm.n_cavities; ++c) e += hm.omega_c * d[L.photon_digit[c]];
        for (size_t a = 0; a < L.atom_digit.size(); ++a) e += hm.omega_a * d[L.atom_digit[a]];
        if (e != 0.0) hm.h_entries.push_back({k, k, e, 0, 0});
        for (size_t a = 0; a < L.atom_digit.size(); ++a) {
            int pa = L.photon_digit[L.atom_cavity[a]], sa = L.atom_digit[a];
            int nph = d[pa], nmax = L.radix[pa] - 1;
            if (d[sa] == 1 && nph < nmax) {          // a^+ sigma
                std::copy(d, d + n, t.begin());
                t[sa] = 0; t[pa] = (uint8_t)(nph + 1);
                emit(k, std::sqrt(nph + 1.0), 1, (int32_t)a);
            }
            if (d[sa] == 0 && nph >= 1) {            // a sigma^+
                std::copy(d, d + n, t.begin());
                t[sa] = 1; t[pa] = (uint8_t)(nph - 1);
                emit(k, std::sqrt((double)nph), 1, (int32_t)a);
            }
        }
        for (size_t b = 0; b < hm.zeta.size(); ++b) {
            int pi = L.photon_digit[hm.bond_i[b]], pj = L.photon_digit[hm.bond_j[b]];
            int ni = d[pi], nj = d[pj];
            if (nj >= 1 && ni < L.radix[pi] - 1) {   // a_i^+ a_j
                std::copy(d, d + n, t.begin());
                t[pi] = (uint8_t)(ni + 1); t[pj] = (uint8_t)(nj - 1);
                emit(k, std::sqrt((ni + 1.0) * nj), 2, (int32_t)b);
            }
            if (ni >= 1 && nj < L.radix[pj] - 1) {   // a_i a_j^+
                std::copy(d, d + n, t.begin());
                t[pi] = (uint8_t)(ni - 1); t[pj] = (uint8_t)(nj + 1);
                emit(k, std::sqrt(ni * (nj + 1.0)), 2, (int32_t)b);
            }
        }
        for (size_t x = 0; x < hm.extra_tunnel.size(); ++x) {
            int px = L.extra_digit[x];
            std::copy(d, d + n, t.begin());
            t[px] = (uint8_t)(1 - d[px]);
            emit(k, 1.0, 3, (int32_t)x);
        }
    }
}

void build_jumps(HostModel &hm) {
    const Layout &L = hm.layout;
    const int n = L.n_digits();
    hm.jumps.clear();
    hm.anti_diag.assign((size_t)hm.dim, 0.0);
    std::vector<uint8_t> t(n);
    std::vector<uint8_t> zero(n, 0);
    int64_t vacuum = find(hm, zero);
    for (size_t j = 0; j < hm.jump_kind.size(); ++j) {
        int kind = hm.jump_kind[j], site = hm.jump_site[j];
        for (int64_t k = 0; k < hm.dim; ++k) {
            const uint8_t *d = &hm.digits[(size_t)k * n];
            int64_t dst = -1;
            double coef = 0.0;
            if (kind == QED_JUMP_A) {
                int p = L.photon_digit[site];
                if (d[p] >= 1) {
                    std::copy(d, d + n, t.begin());
                    t[p] = (uint8_t)(d[p] - 1);
                    dst = find(hm, t);
                    coef = std::sqrt((double)d[p]);
                }
            } else if (kind == QED_JUMP_SIGMA) {
                int p = L.atom_digit[site];
                if (d[p] == 1) {
                    std::copy(d, d + n, t.begin());
                    t[p] = 0;
                    dst = find(hm, t);
                    coef = 1.0;
                }
            } else if (kind == QED_JUMP_DEPHASE) {
                dst = k;
                coef = d[L.extra_digit[site]] == 1 ? 1.0 : -1.0;
            } else if (kind == QED_JUMP_LEAK) {
                int p = L.photon_digit[site];
                int total = 0;
                for (int i = 0; i < n; ++i) total += d[i];
                if (d[p] == 1 && total == 1) {
                    dst = vacuum;
                    coef = 1.0;
                }
            }
            if (dst >= 0) {
                hm.jumps.push_back({(int32_t)j, k, dst, coef});
                hm.anti_diag[(size_t)k] += hm.gamma[j] * coef * coef;
            }
        }
    }
}

}  // namespace

qed_status build_host_model(const qed_spec *spec, HostModel &hm, std::string &err, bool operators) {
    if (!copy_spec(spec, hm, err)) return QED_EINVAL;
    make_layout(hm);
    if (hm.layout.n_digits() == 0) { err = "model has no digits"; return QED_EINVAL; }
    if (!enumerate_basis(hm, err)) return QED_EINVAL;
    if (operators) {
        build_hamiltonian(hm);
        build_jumps(hm);
    }
    return QED_OK;
}

bool restrict_host_model(const HostModel &src, const std::vector<int64_t> &keep, HostModel &dst,
                         std::string &err) {
    const int n = src.layout.n_digits();
    std::vector<int64_t> to_new((size_t)src.dim, -1);
    for (size_t a = 0; a < keep.size(); ++a) {
        const int64_t k = keep[a];
        if (k < 0 || k >= src.dim || (a > 0 && k <= keep[a - 1])) {
            err = "kept indices must be increasing and inside the basis";
            return false;
        }
        to_new[(size_t)k] = (int64_t)a;
    }
    if (keep.empty()) {
        err = "no state kept";
        return false;
    }
    dst = HostModel();
    // the specification, its layout and the parameter tables are unchanged
    dst.n_cavities = src.n_cavities;
    dst.n_extra = src.n_extra;
    dst.basis_kind = src.basis_kind;
    dst.excitation_cap = src.excitation_cap;
    dst.dim_cap = src.dim_cap;
    dst.omega_c = src.omega_c;
    dst.omega_a = src.omega_a;
    dst.atoms_per_cavity = src.atoms_per_cavity;
    dst.n_max = src.n_max;
    dst.g = src.g;
    dst.zeta = src.zeta;
    dst.extra_tunnel = src.extra_tunnel;
    dst.gamma = src.gamma;
    dst.bond_i = src.bond_i;
    dst.bond_j = src.bond_j;
    dst.jump_kind = src.jump_kind;
    dst.jump_site = src.jump_site;
    dst.layout = src.layout;
    dst.dim = (int64_t)keep.size();
    dst.digits.resize((size_t)dst.dim * n);
    dst.index.reserve((size_t)dst.dim * 2);
    for (int64_t a = 0; a < dst.dim; ++a) {
        std::copy(&src.digits[(size_t)keep[(size_t)a] * n], &src.digits[(size_t)keep[(size_t)a] * n] + n,
                  &dst.digits[(size_t)a * n]);
        dst.index.emplace(state_key(&dst.digits[(size_t)a * n], n), a);
    }
    // P H P and P A_j P: the entries between kept states, renumbered
    for (const auto &e : src.h_entries) {
        const int64_t r = to_new[(size_t)e.row], c = to_new[(size_t)e.col];
        if (r >= 0 && c >= 0) dst.h_entries.push_back({r, c, e.unit, e.param, e.which});
    }
    dst.anti_diag.assign((size_t)dst.dim, 0.0);
    for (const auto &e : src.jumps) {
        const int64_t a = to_new[(size_t)e.src], b = to_new[(size_t)e.dst];
        if (a < 0 || b < 0) continue;
        dst.jumps.push_back({e.jump, a, b, e.coef});
        dst.anti_diag[(size_t)a] += dst.gamma[(size_t)e.jump] * e.coef * e.coef;
    }
    return true;
}

double entry_coefficient(const HostModel &hm, const HostModel::HEntry &e) {
    switch (e.param) {
    case 1: return hm.g[e.which];
    case 2: return hm.zeta[e.which];
    case 3: return hm.extra_tunnel[e.which];
    default: return 1.0;
    }
}

void dense_hamiltonian(const HostModel &hm, std::vector<cplx> &H) {
    const int64_t D = hm.dim;
    H.assign((size_t)(D * D), cplx(0.0, 0.0));
    for (const auto &e : hm.h_entries) H[(size_t)(e.row * D + e.col)] += entry_coefficient(hm, e) * e.unit;
}

}  // namespace qed
