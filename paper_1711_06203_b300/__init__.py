"""B300-native CTU-PPM hydro step: CUDA kernels behind a C ABI (libhydro.so)
with a thin ctypes binding.  Importing the package does not load the library;
the binding loads it on first use and fails loudly if it is missing."""
