// Host-side harness for the sanitizer test (built with -fsanitize=address,undefined
// by tests/test_host_sanitize_cpu.py): the host code of the library that runs
// without a GPU, on inputs the test writes and checks.
//   herm_table <in> <out>: in = int32 nR, n; int32 R[nR][3]; float64 X[nR][n][n][2]
//                          out = int32 ok, nrep, M; int32 reps[nrep][3]; float64 T[2 nrep][n*n]
//   heevj <n> <count> <in> <out>: in = float64 mat[count][n][n][2] (Hermitian)
//                          out = float64 eval[count][n], evec[count][n][n][2]
#include <cmath>
#include <cstdint>
#include <cstdio>
#include <cstring>
#include <vector>

#include "heevj.cuh"
#include "herm_table.h"

static bool read_all(const char *path, std::vector<char> &buf) {
    FILE *f = std::fopen(path, "rb");
    if (!f) return false;
    std::fseek(f, 0, SEEK_END);
    const long sz = std::ftell(f);
    std::fseek(f, 0, SEEK_SET);
    buf.resize((size_t)sz);
    const bool ok = std::fread(buf.data(), 1, buf.size(), f) == buf.size();
    std::fclose(f);
    return ok;
}

template <int N>
static void run_heevj(int count, const double *mat, double *eval, double *evec) {
    for (int c = 0; c < count; ++c) {
        double ar[N * N], ai[N * N], vr[N * N], vi[N * N], w[N];
        for (int r = 0; r < N * N; ++r) {
            ar[r] = mat[2 * ((size_t)c * N * N + r)];
            ai[r] = mat[2 * ((size_t)c * N * N + r) + 1];
        }
        pgb::heevj_one<N>(ar, ai, vr, vi, w);
        for (int r = 0; r < N; ++r) eval[(size_t)c * N + r] = w[r];
        for (int r = 0; r < N * N; ++r) {
            evec[2 * ((size_t)c * N * N + r)] = vr[r];
            evec[2 * ((size_t)c * N * N + r) + 1] = vi[r];
        }
    }
}

int main(int argc, char **argv) {
    if (argc == 4 && std::strcmp(argv[1], "herm_table") == 0) {
        std::vector<char> buf;
        if (!read_all(argv[2], buf) || buf.size() < 8) return 2;
        int32_t nR, n;
        std::memcpy(&nR, buf.data(), 4);
        std::memcpy(&n, buf.data() + 4, 4);
        const size_t need = 8 + (size_t)nR * 12 + (size_t)nR * n * n * 16;
        if (nR < 1 || n < 1 || buf.size() != need) return 2;
        std::vector<int32_t> R((size_t)nR * 3);
        std::vector<double> X((size_t)nR * n * n * 2);
        std::memcpy(R.data(), buf.data() + 8, R.size() * 4);
        std::memcpy(X.data(), buf.data() + 8 + R.size() * 4, X.size() * 8);
        std::vector<int32_t> reps;
        std::vector<double> T;
        int M = 0;
        const int32_t ok = pgb::herm_table_host(R.data(), X.data(), nR, n, reps, T, M) ? 1 : 0;
        FILE *f = std::fopen(argv[3], "wb");
        if (!f) return 2;
        const int32_t hdr[3] = {ok, (int32_t)(reps.size() / 3), (int32_t)M};
        std::fwrite(hdr, 4, 3, f);
        if (ok) {
            std::fwrite(reps.data(), 4, reps.size(), f);
            std::fwrite(T.data(), 8, T.size(), f);
        }
        std::fclose(f);
        return 0;
    }
    if (argc == 6 && std::strcmp(argv[1], "heevj") == 0) {
        const int n = std::atoi(argv[2]), count = std::atoi(argv[3]);
        std::vector<char> buf;
        if (!read_all(argv[4], buf) || count < 1 || buf.size() != (size_t)count * n * n * 16) return 2;
        std::vector<double> mat((size_t)count * n * n * 2), eval((size_t)count * n), evec(mat.size());
        std::memcpy(mat.data(), buf.data(), buf.size());
        switch (n) {
            case 2: run_heevj<2>(count, mat.data(), eval.data(), evec.data()); break;
            case 3: run_heevj<3>(count, mat.data(), eval.data(), evec.data()); break;
            case 6: run_heevj<6>(count, mat.data(), eval.data(), evec.data()); break;
            case 8: run_heevj<8>(count, mat.data(), eval.data(), evec.data()); break;
            case 16: run_heevj<16>(count, mat.data(), eval.data(), evec.data()); break;
            default: return 2;
        }
        FILE *f = std::fopen(argv[5], "wb");
        if (!f) return 2;
        std::fwrite(eval.data(), 8, eval.size(), f);
        std::fwrite(evec.data(), 8, evec.size(), f);
        std::fclose(f);
        return 0;
    }
    return 2;
}
