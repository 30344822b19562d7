// Host construction of the modal element coefficients (see modal.cuh).
#include <cmath>
#include <string>

#include "modal.cuh"

namespace topo {

bool build_modal(const double K0[576], ModalCoef* mc, std::string* err) {
    double T[24][24] = {};
    for (int b = 0; b < 8; ++b)
        for (int a = 0; a < 8; ++a) {
            double s = 1.0;
            for (int d = 0; d < 3; ++d)
                if ((b >> d) & 1) s *= ((a >> d) & 1) ? 1.0 : -1.0;
            for (int c = 0; c < 3; ++c) T[3 * b + c][3 * a + c] = s;
        }
    double TK[24][24] = {}, X[24][24] = {};
    for (int i = 0; i < 24; ++i)
        for (int j = 0; j < 24; ++j) {
            double s = 0.0;
            for (int k = 0; k < 24; ++k) s += T[i][k] * K0[k * 24 + j];
            TK[i][j] = s;
        }
    double xmax = 0.0;
    for (int i = 0; i < 24; ++i)
        for (int j = 0; j < 24; ++j) {
            double s = 0.0;
            for (int k = 0; k < 24; ++k) s += TK[i][k] * T[j][k];
            X[i][j] = s / 64.0;
            xmax = std::fmax(xmax, std::fabs(X[i][j]));
        }
    bool pat[24][24] = {};
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            pat[kN(r)][kN(q)] = true;
            pat[kT(r)][kT(q)] = true;
        }
    for (int g = 0; g < 3; ++g)
        for (int r = 0; r < 2; ++r)
            for (int q = 0; q < 2; ++q) {
                pat[kS(g, r)][kS(g, q)] = true;
                pat[kB(g, r)][kB(g, q)] = true;
            }
    for (int r = 0; r < 3; ++r) pat[kC(r)][kC(r)] = true;
    for (int i = 0; i < 24; ++i)
        for (int j = 0; j < 24; ++j)
            if (!pat[i][j] && std::fabs(X[i][j]) > 1e-12 * xmax) {
                if (err) *err = "element matrix lacks the hex8 modal structure at (" + std::to_string(i) + "," +
                                std::to_string(j) + ")";
                return false;
            }
    for (int r = 0; r < 3; ++r)
        for (int q = 0; q < 3; ++q) {
            mc->N[r][q] = X[kN(r)][kN(q)];
            mc->T3[r][q] = X[kT(r)][kT(q)];
        }
    for (int g = 0; g < 3; ++g)
        for (int r = 0; r < 2; ++r)
            for (int q = 0; q < 2; ++q) {
                mc->S[g][r][q] = X[kS(g, r)][kS(g, q)];
                mc->B[g][r][q] = X[kB(g, r)][kB(g, q)];
            }
    for (int r = 0; r < 3; ++r) mc->C[r] = X[kC(r)][kC(r)];
    return true;
}

}  // namespace topo
