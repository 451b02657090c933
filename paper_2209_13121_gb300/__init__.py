"""GB300-native P-RSoXS forward model (Algorithm 1 hot path).

Importing the package does not load the CUDA library; `paper_2209_13121_gb300.rsx`
does, and fails loudly when it is missing."""
