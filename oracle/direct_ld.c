/*
 * The direct-sum oracle of direct.c in extended precision (long double:
 * 64-bit significand on x86, binary128 where the platform's long double is),
 * exported with the suffix _ld.  TEST INFRASTRUCTURE ONLY.
 */
#define REAL long double
#define SUFFIX(name) name##_ld
#include "direct.c"
