"""FP64 CPU oracle of the optical-flow FEM system (test infrastructure only:
imported by the tests, the package smoke check and the benchmark's CPU
baseline, never by the product path)."""
