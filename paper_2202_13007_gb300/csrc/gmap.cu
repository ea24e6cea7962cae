// gmap.cu -- host computation of the decompression map G (see gmap.cuh).
#include <cmath>
#include <mutex>

#include "gmap.cuh"

namespace blaz {

const long double (*decompress_map())[kKeep]
{
    static long double G[64][kKeep];
    static std::once_flag once;
    std::call_once(once, [] {
        const long double pi = 3.14159265358979323846264338327950288L;
        long double c[8][8];
        for (int k = 0; k < 8; ++k)
            for (int x = 0; x < 8; ++x) c[k][x] = cosl((long double)((2 * x + 1) * k) * pi / 16.0L);
        const long double al[8] = {sqrtl(0.125L), 0.5L, 0.5L, 0.5L, 0.5L, 0.5L, 0.5L, 0.5L};
        for (int t = 0; t < kKeep; ++t) {
            const int i = kept_row(t), j = kept_col(t);
            long double B[8][8];
            for (int u = 0; u < 8; ++u)
                for (int v = 0; v < 8; ++v) {
                    const long double P = al[i] * al[j] * c[i][u] * c[j][v];
                    if (u == 0 && v == 0) B[u][v] = 0.0L;
                    else if (u == 0) B[u][v] = B[u][v - 1] + P;
                    else if (v == 0) B[u][v] = B[u - 1][v] + P;
                    else B[u][v] = (B[u - 1][v] + B[u][v - 1]) * 0.5L + P;
                    G[u * 8 + v][t] = B[u][v];
                }
        }
    });
    return G;
}

}  // namespace blaz
