// Host-side model data (factors of a discrete graphical model).
#pragma once
#include <cstdint>
#include <string>
#include <vector>

namespace tn {

struct ModelData {
    int nvars = 0;
    std::vector<int> card;
    int nfactors = 0;
    std::vector<std::vector<int>> scope;   // storage order, last fastest
    std::vector<int64_t> toff;             // table offset of each factor
    std::vector<double> tables;
};

std::string validate_model(const ModelData &m);
std::string model_from_arrays(int nvars, const int *card, int nfactors, const int *scope_off,
                              const int *scope_vars, const double *tables, ModelData &m);
std::string model_from_uai(const char *path, ModelData &m, bool &parse_error);
// UAI evidence file: "<nobs> v1 x1 ... " (one evidence set) or "<nsets>"
// followed by nsets such blocks; each set becomes a row over all variables
// (-1 = unobserved).
std::string evidence_from_uai(const char *path, const ModelData &m,
                              std::vector<std::vector<int32_t>> &sets, bool &parse_error);
// UAI MMAP query file: "<nq> v1 ... vq".
std::string query_from_uai(const char *path, const ModelData &m, std::vector<int32_t> &q,
                           bool &parse_error);

}  // namespace tn
