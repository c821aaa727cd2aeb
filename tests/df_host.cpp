// Host driver for the double-float arithmetic of csrc/df.cuh (compiled by
// tests/test_df_host.py with the host compiler): reads lines
// "op a b" with a, b doubles in hexadecimal floating notation and prints,
// per line, the double-float operands and result as hexadecimal floats
// (a.hi a.lo b.hi b.lo r.hi r.lo), so that the test can check each step
// against exact rational arithmetic.
#include <cstdio>
#include <cstdlib>
#include <cstring>

#include "df.cuh"

int main() {
    char op[16];
    double a, b;
    while (std::scanf("%15s %la %la", op, &a, &b) == 3) {
        const dda::DF x(a), y(b);
        dda::DF r;
        if (!std::strcmp(op, "add")) r = x + y;
        else if (!std::strcmp(op, "sub")) r = x - y;
        else if (!std::strcmp(op, "mul")) r = x * y;
        else if (!std::strcmp(op, "fma")) r = dda::fma(x, y, x);
        else if (!std::strcmp(op, "two_sum")) r = dda::df_two_sum((float)a, (float)b);
        else return 2;
        std::printf("%a %a %a %a %a %a\n", (double)x.hi, (double)x.lo, (double)y.hi, (double)y.lo, (double)r.hi,
                    (double)r.lo);
    }
    return 0;
}
