"""B300-native SGP4 near-Earth propagation (see include/sgp4.h for the C ABI)."""
