"""GB300-native split-operator Dirac stepper (placeholder; binding added with the library)."""
